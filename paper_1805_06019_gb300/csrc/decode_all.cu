// Full light-field decode: Algorithm 2 for every (view, block location).
//
// One CTA owns a strip of kNL consecutive block locations of one block row.
// Its 3 * kNL records (location-major, then Y / Co / Cg) are contiguous in the
// stream; they are copied into shared memory when they fit the CTA's staging
// budget and read from the stream otherwise.  Phases:
//  1. parse (a warp per record): each record's presence mask, the
//     stored-block count in front of each mask word, and the payload bit
//     offset of every stored block (closed-form lengths of the 18-bit
//     headers, warp scan), in one compact table for the strip;
//  2. internal nodes (levels >= 1, first in BFS order), level by level from
//     the top, a thread per (location, node, channel): the reconstruction is
//     the parent reconstruction (or top RKV) plus the decoded residual where
//     a block is stored; then a thread per (location, parent, block row)
//     converts the view parents' rows to RGB.  Barriers separate these steps.
//     The last warp also prefetches into L2 the records and top-RKV blocks
//     of the strip a CTA of the next wave will take; then
//  3. the views, one unit of kUnit (8) BFS positions at a time per warp
//     (each warp takes the next unit from a shared counter and never waits
//     for the others).  The unit's output rows (8 views x 4 block rows x
//     the strip's 96 bytes) are assembled in the warp's shared-memory
//     buffer and written once:
//     a. the buffer starts as every view's parent rows (RGB), the exact
//        result for every block without a stored residual (most of them);
//     b. the unit's items (a view's block with at least one stored channel)
//        and slots (a stored channel block): lane = (view, quarter of the
//        strip) reads the three channel masks of its two locations, and one
//        warp scan of the per-lane counts places every item and slot; lanes
//        whose slots do not fit the warp's kWSlots decode slots go in a
//        further run.  Every slot is decoded by one lane (a mode-generic
//        BISE decoder that builds two values per multiply-add, see
//        decode_block_pairs); then four lanes per item, one block row each,
//        add the residual rows to the parent rows, apply the inverse
//        YCoCg-R two pixels per instruction and overwrite the item's bytes
//        in the buffer;
//     c. the buffer is written as whole 16-byte chunks, consecutive lanes
//        on consecutive chunks of one view row (one large L2 write per view
//        row instead of one per block row).
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
constexpr int kThreads = 384;                    // twelve warps: eight parse the strip's locations, all twelve take view units
constexpr int kWarps = kThreads / 32;
constexpr int kUnit = 8;                         // BFS positions per unit of view work (a quarter mask word)
constexpr int kWSlots = 32;                      // decode slots per warp
constexpr int kZeroSlot = kWSlots;               // a slot of zero residuals, for channels without a stored block
constexpr int kWItems = kNL * kUnit;             // items per warp at most (every block of a unit)
constexpr uint32_t kSmemBudget = 200 * 1024;
constexpr size_t kCtaSmemTarget = 111 * 1024;    // two CTAs per SM (with the static arrays and the 1 KB each CTA reserves): staging fills up to this
constexpr uint32_t kNodeSmemMax = 4096;          // node tables up to this size are cached per CTA

static_assert(kNL == 8, "the location and group splits below assume eight locations per strip");
static_assert(3 * kNL <= 32 && (kNL & (kNL - 1)) == 0, "the strip's records fit one warp's lanes; locations are a power of two");
static_assert(kUnit == 8, "a unit is a quarter of a 32-bit mask word");
static_assert(kNL == 8 && kUnit * 4 == 32, "the list builder's lanes are (view of the unit, quarter of the strip)");
static_assert(kWSlots >= 6, "one lane's slots (two locations, three channels) must fit a run");

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
    uint32_t vec16;          // a strip's view rows go out as whole 16-byte chunks (16-byte aligned output; RGB: W % 16 == 0, packed: W % 4 == 0)
    uint32_t vec4;           // where they cannot, as 4-byte words (4-byte aligned output; RGB also W % 4 == 0)
    uint32_t pmax;           // largest number of stored blocks in the records of one strip
    uint32_t n_units;        // ceil(S / kUnit)
    uint32_t node_smem;      // the node table is cached in shared memory
    uint32_t stage_words;    // shared-memory words for the strip's records (0: read them from the stream)
    uint32_t lvl_begin[kMaxLevels];  // first BFS position of each internal level, top level first; [L-2] = n_int
    uint32_t *dbg;           // debug builds: the stream's flag word
    uint32_t n_out;          // output views (or slots of the packed instantiation)
    uint32_t ahead;          // CTAs resident at once: the strip this many ahead is prefetched into L2
};

template <bool kPacked>
__host__ __device__ constexpr uint32_t row_words() { return kPacked ? 4u : 3u; }
// one warp's output buffer, in 16-byte chunks: kUnit views x 4 rows x kNL locations x row_words
template <bool kPacked>
__host__ __device__ constexpr uint32_t obuf_words() { return kUnit * 4 * kNL * row_words<kPacked>() / 4; }

struct Smem {
    uint32_t *slots;   // [warp][kWSlots + 1][8]  decoded blocks, biased pairs; slot kZeroSlot is zero
    uint32_t *top;     // [n_top][kNL][24]  biased pairs
    uint32_t *inter;   // [n_int][kNL][24]  internal reconstructions, biased pairs
    uint32_t *mask;    // [kRecs][MW]
    uint32_t *mpre;    // [kRecs][MW]  stored blocks in front of each mask word
    uint32_t *need;    // [MW]  views to decode (bit per BFS position)
    uint32_t *node;    // [S]  node table (when cached)
    uint32_t *sent;    // [warp][kWSlots]  record | rank << 8
    uint32_t *items;   // [warp][kWItems]  p | l << 14 | stored channels << 18 | first slot << 21
    uint32_t *obuf;    // [warp][kUnit][4][kNL * 4 * bytes per pixel]  the unit's output rows
    uint32_t *prgb;    // [n_par][4][kNL][row_words]  parent rows converted to RGB
    void *off;         // [pmax]  payload bit offset of each stored block (OffT), record after record
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
    s.top = reinterpret_cast<uint32_t *>(take(96ull * a.n_top * kNL));
    s.inter = reinterpret_cast<uint32_t *>(take(96ull * a.n_int * kNL));
    s.mask = reinterpret_cast<uint32_t *>(take(4ull * kRecs * a.MW));
    s.mpre = reinterpret_cast<uint32_t *>(take(4ull * kRecs * a.MW));
    s.need = reinterpret_cast<uint32_t *>(take(4ull * a.MW));
    s.node = reinterpret_cast<uint32_t *>(take(a.node_smem ? 4ull * a.S : 0));
    s.sent = reinterpret_cast<uint32_t *>(take(4ull * kWSlots * kWarps));
    s.items = reinterpret_cast<uint32_t *>(take(4ull * kWItems * kWarps));
    s.obuf = reinterpret_cast<uint32_t *>(take(16ull * obuf_words<kPacked>() * kWarps));
    s.prgb = reinterpret_cast<uint32_t *>(take(16ull * row_words<kPacked>() * a.n_par * kNL));
    s.off = take(off_size * a.pmax);
    s.stage = reinterpret_cast<uint32_t *>(take(4ull * a.stage_words));
    if (m)
        *m = s;
    return at;
}

// ---- one BISE block, any mode, by one thread ---------------------------------
//
// The 16 values come out dequantised and biased, two to a word (value 2j in
// the low half of out[j], 2j + 1 in the high half), and are built two at a
// time: every term of (digit << b | low part) << shift + (min << shift) +
// 2^14 is non-negative and the sum of each half stays below 2^15 (the
// loader's range check), so the pair needs one 32-bit multiply-add per term
// and no carry crosses the halves.
// Digits (trit and quint blocks) come first in the payload: the groups are
// split by the base-3 / base-5 tables (digit v at bits 3v of a 64-bit word).
// The low parts of block row rr (values 4rr .. 4rr + 3, 4b <= 40 bits) sit
// in one 64-bit window of the payload read from three record words.
__device__ __forceinline__ void decode_block_pairs(const uint32_t *rec, uint32_t pos, uint32_t hdr, uint32_t q,
                                                   const uint32_t *s_mode, const uint16_t *s_dig, uint32_t out[8])
{
    const uint32_t mp = s_mode[hdr & 31u];
    const uint32_t b = mode_b(mp), kind = mode_kind(mp);
    const uint32_t scale = 1u << (q + ((hdr >> 5) & 3u));
    const int32_t mn = ((int32_t)(hdr << 14)) >> 21;   // header bits 7..17, sign-extended
    const uint32_t base = (uint32_t)mn * scale + 0x4000u;
    const uint32_t base2 = base | (base << 16);
    const uint32_t m2 = ((1u << b) - 1u) * 0x10001u;   // the low-part mask in both halves
    const uint32_t sb = scale << b;
    uint64_t dw = 0;   // digit v at bits 3v
    uint32_t D = 0;    // digit bits in front of the low parts
    if (kind != 0) {
        const uint32_t *w = rec + (pos >> 5);
        const uint32_t x0 = w[0], x1 = w[1], x2 = w[2];
        const uint32_t A0 = __funnelshift_r(x0, x1, pos), A1 = __funnelshift_r(x1, x2, pos);
        if (kind == 1) {
            // trits: three 8-bit digit groups and a 2-bit one (value 15), low parts from bit 26
            uint32_t t3 = (A0 >> 24) & 3u;
            t3 = t3 == 3u ? 0u : t3;
            dw = (uint64_t)s_dig[A0 & 0xFFu] | ((uint64_t)s_dig[(A0 >> 8) & 0xFFu] << 15) |
                 ((uint64_t)s_dig[(A0 >> 16) & 0xFFu] << 30) | ((uint64_t)t3 << 45);
            D = 26;
        } else {
            // quints: five 7-bit digit groups and a 3-bit one (value 15), low parts from bit 38
            uint32_t t5 = (A1 >> 3) & 7u;
            t5 = t5 >= 5u ? t5 - 5u : t5;
            dw = (uint64_t)s_dig[256u + (A0 & 0x7Fu)] | ((uint64_t)s_dig[256u + ((A0 >> 7) & 0x7Fu)] << 9) |
                 ((uint64_t)s_dig[256u + ((A0 >> 14) & 0x7Fu)] << 18) |
                 ((uint64_t)s_dig[256u + ((A0 >> 21) & 0x7Fu)] << 27) |
                 ((uint64_t)s_dig[256u + (__funnelshift_r(A0, A1, 28) & 0x7Fu)] << 36) | ((uint64_t)t5 << 45);
            D = 38;
        }
    }
#pragma unroll
    for (uint32_t rr = 0; rr < 4; rr++) {
        const uint32_t lp = pos + D + 4u * rr * b;   // the row's first low part
        const uint32_t *w = rec + (lp >> 5);
        const uint32_t y0 = w[0], y1 = w[1], y2 = w[2];
        const uint32_t lo = __funnelshift_r(y0, y1, lp), hi = __funnelshift_r(y1, y2, lp);
        // low parts of values (0, 1) and (2, 3) of the row, one per half (shifts <= 3b <= 30)
        const uint32_t l01 = __byte_perm(lo, __funnelshift_r(lo, hi, b), 0x5410) & m2;
        const uint32_t l23 = __byte_perm(__funnelshift_r(lo, hi, 2 * b), __funnelshift_r(lo, hi, 3 * b), 0x5410) & m2;
        // digits of the row: 12 bits; d * (1 + 2^13) puts digit 1 at bit 16
        const uint32_t dr = (uint32_t)(dw >> (12 * rr)) & 0xFFFu;
        const uint32_t d01 = (dr * 0x2001u) & 0x70007u, d23 = ((dr >> 6) * 0x2001u) & 0x70007u;
        out[2 * rr] = d01 * sb + l01 * scale + base2;
        out[2 * rr + 1] = d23 * sb + l23 * scale + base2;
    }
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

// Address of pixel (x, y) of output view slot ov.
template <bool kPacked>
__device__ __forceinline__ uint8_t *out_px(const Args &a, uint32_t ov, uint32_t y, uint32_t x)
{
    return a.out + (((size_t)ov * a.H + y) * a.W + x) * (kPacked ? 4u : 3u);
}

template <bool kPacked, typename OffT>
__global__ void __launch_bounds__(kThreads, 2) decode_all_kernel(const Args a)
{
    __shared__ uint32_t s_mode[32];
    __shared__ uint16_t s_dig[256 + 128];
    __shared__ uint32_t s_roff[kRecs];
    __shared__ uint32_t s_np[kRecs];      // stored blocks of each record of the strip
    __shared__ uint32_t s_obase[kRecs];   // where each record's payload offsets start in m_off
#ifdef RLFC_DEBUG
    __shared__ uint32_t s_rbits[kRecs];   // length of each record in bits
#endif
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
    // the records of the strip a CTA of the next wave will take: the last
    // warp loads their range now and prefetches them into L2 once the parse
    // is done, so that CTA's staging reads hit L2 instead of DRAM
    uint32_t pf_lo = 0, pf_hi = 0, pf_top = 0xFFFFFFFFu, pf_nl = 0;   // pf_top, pf_nl: the strip's first location and count
    {
        const uint32_t strip2 = blockIdx.y * gridDim.x + blockIdx.x + a.ahead;
        if (warp == kWarps - 1 && a.ahead && strip2 < gridDim.x * gridDim.y) {
            const uint32_t bx2 = (strip2 % gridDim.x) * kNL, b02 = (strip2 / gridDim.x) * a.nlx + bx2;
            const uint32_t nl2 = min((uint32_t)kNL, a.nlx - bx2);
            pf_lo = __ldg(a.offsets + 3 * b02) & ~31u;
            pf_hi = __ldg(a.offsets + 3 * (b02 + nl2));
            pf_top = b02;
            pf_nl = nl2;
        }
    }
#ifdef RLFC_DEBUG
    if (tid < kRecs)
        s_rbits[tid] = tid < 3 * (int)nl ? 32u * (__ldg(a.offsets + 3 * b0 + tid + 1) - __ldg(a.offsets + 3 * b0 + tid)) : 0u;
#endif
    {
        const uint32_t *tg = reinterpret_cast<const uint32_t *>(a.top);
        for (uint32_t i = tid; i < a.n_top * kNL * 24; i += kThreads) {
            const uint32_t t = i / (kNL * 24), rest = i - t * (kNL * 24), loc = rest / 24, wi = rest - loc * 24;
            m.top[i] = loc < nl ? (__ldg(tg + ((size_t)t * a.nloc + b0 + loc) * 24 + wi) ^ 0x80008000u) - kB2 : kB2;
        }
    }
    uint32_t *wslots = m.slots + warp * (8 * (kWSlots + 1));   // this warp's slots
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

    // ---- phases 1 and 2, spread over all warps: parse the strip's records
    // (a warp per record), reconstruct the internal nodes level by level (a
    // thread per (location, node, channel)), convert the view parents' rows
    // to RGB (a thread per (location, parent, block row))
    const uint32_t hdr0 = 32 * a.MW;
    // 1a. per record: mask words and the stored blocks in front of each
    // (nothing stored past the end of the row)
    for (uint32_t r = warp; r < (uint32_t)kRecs; r += kWarps) {
        const bool live = r < 3 * nl;
        uint32_t *mk = m.mask + r * a.MW;
        uint32_t *mp = m.mpre + r * a.MW;
        const uint32_t *rec = rb + s_roff[r];
        uint32_t P = 0;
        for (uint32_t w0 = 0; w0 < a.MW; w0 += 32) {
            const uint32_t word = (live && w0 + lane < a.MW) ? rec[w0 + lane] : 0u;
            const uint32_t cnt = (uint32_t)__popc(word);
            const uint32_t incl = warp_inclusive_scan(cnt, lane);
            if (w0 + lane < a.MW) {
                mk[w0 + lane] = word;
                mp[w0 + lane] = P + incl - cnt;
            }
            P += __shfl_sync(kFullMask, incl, 31);
        }
        if (lane == 0)
            s_np[r] = P;
    }
    __syncthreads();
    // the strip's payload offsets go record after record into m_off
    const uint32_t np_l = lane < kRecs ? s_np[lane] : 0u;
    const uint32_t ob_l = warp_inclusive_scan(np_l, lane) - np_l;
    if (warp == 0 && lane < kRecs)
        s_obase[lane] = ob_l;
    // 1b. per record: payload offset of every stored block (closed-form
    // lengths of the 18-bit headers, warp scan)
    for (uint32_t r = warp; r < 3 * nl; r += kWarps) {
        const uint32_t *rec = rb + s_roff[r];
        const uint32_t P = s_np[r];
        OffT *o = m_off + __shfl_sync(kFullMask, ob_l, r);
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
                o[h] = (OffT)(run + incl - len);
            run += __shfl_sync(kFullMask, incl, 31);
        }
    }
    __syncthreads();
    // 2. internal nodes, level by level from the top: reconstruction =
    // parent reconstruction (top RKV or a node of the level above) + the
    // decoded residual where a block is stored
    for (uint32_t lv = 0; lv + 2 < a.L; lv++) {
        const uint32_t g0 = a.lvl_begin[lv], g1 = a.lvl_begin[lv + 1];
        const uint32_t *src = lv == 0 ? m.top : m.inter;
        for (uint32_t t = tid; t < (g1 - g0) * 3 * kNL; t += kThreads) {
            const uint32_t l = t & (kNL - 1), q = t / kNL;
            if (l >= nl)
                continue;
            const uint32_t p = g0 + q / 3, c = q - 3 * (q / 3), r = 3 * l + c;
            const uint32_t word = m.mask[r * a.MW + (p >> 5)];
            uint32_t v[8];
            if ((word >> (p & 31u)) & 1u) {
                const uint32_t rank = m.mpre[r * a.MW + (p >> 5)] + __popc(word & ((1u << (p & 31u)) - 1u));
                const uint32_t *rec = rb + s_roff[r];
                const uint32_t bp = hdr0 + kHdrBits * rank;
                const uint32_t hdr = __funnelshift_r(rec[bp >> 5], rec[(bp >> 5) + 1], bp) & 0x3FFFFu;
                const uint32_t pos = m_off[s_obase[r] + rank];
#ifdef RLFC_DEBUG
                if (RLFC_DBG_BLOCK_OK(a.dbg, hdr & 31u, bp + kHdrBits, hdr0 + kHdrBits * s_np[r], pos,
                                      (hdr & 31u) < (uint32_t)kNumModes ? mode_bits(s_mode[hdr & 31u]) : 0u,
                                      s_rbits[r]))
                    decode_block_pairs(rec, pos, hdr, a.q, s_mode, s_dig, v);
                else
                    for (int j = 0; j < 8; j++)
                        v[j] = kB2;
#else
                decode_block_pairs(rec, pos, hdr, a.q, s_mode, s_dig, v);
#endif
            } else {
#pragma unroll
                for (int j = 0; j < 8; j++)
                    v[j] = kB2;
            }
            const uint4 *ps = reinterpret_cast<const uint4 *>(src + (node_parent(nodes[p]) * kNL + l) * 24 + c * 8);
            uint4 *pd = reinterpret_cast<uint4 *>(m.inter + (p * kNL + l) * 24 + c * 8);
            const uint4 s0 = ps[0], s1 = ps[1];
            pd[0] = make_uint4(s0.x + v[0] - kB2, s0.y + v[1] - kB2, s0.z + v[2] - kB2, s0.w + v[3] - kB2);
            pd[1] = make_uint4(s1.x + v[4] - kB2, s1.y + v[5] - kB2, s1.z + v[6] - kB2, s1.w + v[7] - kB2);
        }
        __syncthreads();
    }
    // 3. the block rows of every parent of a view, as RGB
    {
        const uint32_t *src = a.L == 2 ? m.top : m.inter;
        for (uint32_t t = tid; t < a.n_par * 4 * kNL; t += kThreads) {
            const uint32_t l = t & (kNL - 1), q = t / kNL, n = q >> 2, rr = q & 3u;
            if (l >= nl)
                continue;
            const uint32_t *sl = src + ((a.par_base + n) * kNL + l) * 24 + rr * 2;
            uint32_t w[4];
            row_to_rgb<kPacked>(*reinterpret_cast<const uint2 *>(sl), *reinterpret_cast<const uint2 *>(sl + 8),
                                *reinterpret_cast<const uint2 *>(sl + 16), w);
            uint32_t *d = m.prgb + ((n * 4 + rr) * kNL + l) * RW;
#pragma unroll
            for (uint32_t k = 0; k < RW; k++)
                d[k] = w[k];
        }
    }
    __syncthreads();
    if (warp == kWarps - 1) {
        for (uint32_t i = pf_lo + 32u * lane; i < pf_hi; i += 32u * 32u)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(__cvta_generic_to_global(a.records + i)));
        // the strip's top-RKV blocks: 96 bytes per location, per top RKV
        if (pf_top != 0xFFFFFFFFu && lane < (int)a.n_top * 6 && (lane % 6) * 64 < pf_nl * 48)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(__cvta_generic_to_global(
                a.top + ((size_t)(lane / 6) * a.nloc + pf_top) * 48 + (lane % 6) * 64)));
    }

    // ---- phase 3: the views, one unit of kUnit positions at a time per warp.
    // The unit's output rows (kUnit views x 4 rows x the strip's kNL
    // locations) are assembled in the warp's buffer, then written once, each
    // view row as whole 16-byte chunks by consecutive lanes: few, large L2
    // writes instead of one per block row.
    const uint32_t *par_slab = a.L == 2 ? m.top : m.inter;
    const uint32_t u_first = a.n_int / kUnit;
    const uint32_t nrows = min(4u, a.H - by * 4);
    constexpr uint32_t BPP = kPacked ? 4u : 3u;     // output bytes per pixel
    constexpr uint32_t CH = kNL * 4 * BPP / 16;     // 16-byte chunks per view row of the strip
    uint4 *wbuf = reinterpret_cast<uint4 *>(m.obuf) + warp * obuf_words<kPacked>();
    // a strip row written as whole chunks: every location present and 16-byte aligned rows
    const bool whole = a.vec16 && nl == (uint32_t)kNL;
    // otherwise the strip row's bytes (the image may end inside the strip)
    const uint32_t piece = min(nl * 4u, a.W - bx0 * 4u) * BPP;
    for (;;) {
        uint32_t u = 0;
        if (lane == 0)
            u = atomicAdd(&s_unit, 1u);
        u = __shfl_sync(kFullMask, u, 0) + u_first;
        if (u >= a.n_units)
            break;
        const uint32_t w = u >> 2, ub = kUnit * (u & 3u);   // the unit is bits [ub, ub + 8) of mask word w
        const uint32_t P0 = max(u * kUnit, a.n_int), P1 = min(u * kUnit + kUnit, a.S);
        const uint32_t lo = P0 - w * 32, hi = P1 - w * 32;
        const uint32_t sel = (hi >= 32 ? 0xFFFFFFFFu : ((1u << hi) - 1u)) & ~((1u << lo) - 1u) & m.need[w];
        // per view of the unit (lane v < kUnit): its parent's rows and its
        // output rows
        uint32_t par_v = 0;
        uint8_t *out_v = a.out;
        if ((uint32_t)lane < (uint32_t)kUnit && ((sel >> (ub + lane)) & 1u)) {
            const uint32_t info = nodes[w * 32 + ub + lane];
            par_v = (node_parent(info) - a.par_base) * 4 * CH;
            const uint32_t ov = a.slot_of ? __ldg(a.slot_of + node_view(info)) : node_view(info);
            out_v = RLFC_DBG_INDEX_OK(a.dbg, ov, a.n_out) ? out_px<kPacked>(a, ov, by * 4, bx0 * 4) : nullptr;
        }
        // (a) the buffer starts as every view's parent rows (RGB), the exact
        // result for every block without a stored residual; lane = (row,
        // chunk of the view row)
        const uint32_t f_rr = (uint32_t)lane / CH, f_c = (uint32_t)lane % CH;
        const bool f_act = (uint32_t)lane < 4 * CH;
#pragma unroll
        for (uint32_t vv = 0; vv < (uint32_t)kUnit; vv++) {
            const uint32_t pv = __shfl_sync(kFullMask, par_v, vv);
            if (((sel >> (ub + vv)) & 1u) && f_act)
                wbuf[vv * 4 * CH + lane] = reinterpret_cast<const uint4 *>(m.prgb)[pv + lane];
        }
        // (b) items and slots.  Lane = (view ub + v, quarter qd of the strip):
        // the stored channels of its two locations 2qd, 2qd + 1
        const uint32_t v = (uint32_t)lane & 7u, qd = (uint32_t)lane >> 3, bit = ub + v;
        const uint32_t lt = (1u << bit) - 1u;   // positions in front of this view in mask word w
        const bool vsel = (sel >> bit) & 1u;
        uint32_t f[2][3];   // channel masks (word w) of the lane's locations
        uint32_t st = 0;    // stored channels of location 2qd + j at bits 3j .. 3j + 2
        uint32_t ni = 0, ns = 0;
#pragma unroll
        for (uint32_t j = 0; j < 2; j++) {
            const uint32_t l = 2u * qd + j;
#pragma unroll
            for (uint32_t c = 0; c < 3; c++)
                f[j][c] = m.mask[(3 * l + c) * a.MW + w];
            const uint32_t s3 = vsel ? (((f[j][0] >> bit) & 1u) | (((f[j][1] >> bit) & 1u) << 1) |
                                        (((f[j][2] >> bit) & 1u) << 2))
                                     : 0u;
            st |= s3 << (3 * j);
            ni += s3 != 0;
            ns += (uint32_t)__popc(s3);
        }
        const uint32_t cnt = ni | (ns << 16);
        const uint32_t incl = warp_inclusive_scan(cnt, lane);
        const uint32_t excl = incl - cnt;
        __syncwarp();
        // runs of lanes whose slots fit the warp's kWSlots (one lane has at most 6)
        for (uint32_t L0 = 0; L0 < 32;) {
            const uint32_t rb_i = __shfl_sync(kFullMask, excl & 0xFFFFu, L0);
            const uint32_t rb_s = __shfl_sync(kFullMask, excl >> 16, L0);
            const unsigned fit = __ballot_sync(kFullMask, (uint32_t)lane >= L0 && (incl >> 16) - rb_s <= (uint32_t)kWSlots);
            const uint32_t L1 = 32u - (uint32_t)__clz(fit);
            const uint32_t tot = __shfl_sync(kFullMask, incl, L1 - 1);
            const uint32_t n_items = (tot & 0xFFFFu) - rb_i, n_slots = (tot >> 16) - rb_s;
            if ((uint32_t)lane >= L0 && (uint32_t)lane < L1 && st) {
                uint32_t item = (excl & 0xFFFFu) - rb_i, slot = (excl >> 16) - rb_s;
#pragma unroll
                for (uint32_t j = 0; j < 2; j++) {
                    const uint32_t s3 = (st >> (3 * j)) & 7u, l = 2u * qd + j;
                    if (s3) {
                        witems[item++] = (w * 32 + bit) | (l << 14) | (s3 << 18) | (slot << 21);
#pragma unroll
                        for (uint32_t c = 0; c < 3; c++)
                            if ((s3 >> c) & 1u) {
                                const uint32_t r = 3 * l + c;
                                wsent[slot++] = r | ((m.mpre[r * a.MW + w] + __popc(f[j][c] & lt)) << 8);
                            }
                    }
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
                uint32_t dv[8];
#ifdef RLFC_DEBUG
                const uint32_t pos = m_off[s_obase[r] + rank];
                if (RLFC_DBG_BLOCK_OK(a.dbg, hdr & 31u, bp + kHdrBits, hdr0 + kHdrBits * s_np[r], pos,
                                      (hdr & 31u) < (uint32_t)kNumModes ? mode_bits(s_mode[hdr & 31u]) : 0u,
                                      s_rbits[r]))
                    decode_block_pairs(rec, pos, hdr, a.q, s_mode, s_dig, dv);
                else
                    for (int j = 0; j < 8; j++)
                        dv[j] = kB2;
#else
                decode_block_pairs(rec, m_off[s_obase[r] + rank], hdr, a.q, s_mode, s_dig, dv);
#endif
                uint4 *d = reinterpret_cast<uint4 *>(wslots + t * 8);
                d[0] = make_uint4(dv[0], dv[1], dv[2], dv[3]);
                d[1] = make_uint4(dv[4], dv[5], dv[6], dv[7]);
            }
            __syncwarp();
            // items: parent + residual -> RGB into the buffer, four lanes per item, one block row each
            for (uint32_t t = lane; t < 4 * n_items; t += 32) {
                const uint32_t it = witems[t >> 2], rr = t & 3u;
                const uint32_t p = it & 0x3FFFu, l = (it >> 14) & 15u, s3 = (it >> 18) & 7u, s0 = it >> 21;
                const uint32_t *ps = par_slab + (node_parent(nodes[p]) * kNL + l) * 24 + 2 * rr;
                // slot of each channel's residual, or the zero slot
                const uint32_t *ry = wslots + 8 * ((s3 & 1u) ? s0 : (uint32_t)kZeroSlot) + 2 * rr;
                const uint32_t *rco = wslots + 8 * ((s3 & 2u) ? s0 + (s3 & 1u) : (uint32_t)kZeroSlot) + 2 * rr;
                const uint32_t *rcg = wslots + 8 * ((s3 & 4u) ? s0 + __popc(s3 & 3u) : (uint32_t)kZeroSlot) + 2 * rr;
                const uint2 py = *reinterpret_cast<const uint2 *>(ps);
                const uint2 pco = *reinterpret_cast<const uint2 *>(ps + 8);
                const uint2 pcg = *reinterpret_cast<const uint2 *>(ps + 16);
                const uint2 vy = *reinterpret_cast<const uint2 *>(ry);
                const uint2 vco = *reinterpret_cast<const uint2 *>(rco);
                const uint2 vcg = *reinterpret_cast<const uint2 *>(rcg);
                uint32_t wv[4];
                row_to_rgb<kPacked>(make_uint2(py.x + vy.x - kB2, py.y + vy.y - kB2),
                                    make_uint2(pco.x + vco.x - kB2, pco.y + vco.y - kB2),
                                    make_uint2(pcg.x + vcg.x - kB2, pcg.y + vcg.y - kB2), wv);
                uint32_t *d = reinterpret_cast<uint32_t *>(wbuf) + ((p - w * 32 - ub) * 4 + rr) * (kNL * RW) + l * RW;
#pragma unroll
                for (uint32_t k = 0; k < RW; k++)
                    d[k] = wv[k];
            }
            __syncwarp();
            L0 = L1;
        }
        // (c) write the unit's rows: consecutive lanes, consecutive chunks of one view row
        if (whole) {
            const size_t row_bytes = (size_t)a.W * BPP;
#pragma unroll
            for (uint32_t vv = 0; vv < (uint32_t)kUnit; vv++) {
                uint8_t *o = reinterpret_cast<uint8_t *>(
                    __shfl_sync(kFullMask, reinterpret_cast<unsigned long long>(out_v), vv));
                if (((sel >> (ub + vv)) & 1u) && f_act && f_rr < nrows && o)
                    reinterpret_cast<uint4 *>(o + f_rr * row_bytes)[f_c] = wbuf[vv * 4 * CH + lane];
            }
        } else {
            // the right edge of the image, or rows not 16-byte aligned: 4-byte
            // words where the rows allow, else bytes
            const uint8_t *bb = reinterpret_cast<const uint8_t *>(wbuf);
            const uint32_t unit = (a.vec4 && piece % 4 == 0) ? 4u : 1u, per = piece / unit;
            for (uint32_t i = lane; i < kUnit * 4 * per; i += 32) {
                const uint32_t vv = i / (4 * per), rr = (i / per) & 3u, k = i % per;
                const uint32_t view = ((sel >> (ub + vv)) & 1u) ? node_view(nodes[w * 32 + ub + vv]) : 0u;
                const uint32_t ov = ((sel >> (ub + vv)) & 1u) ? (a.slot_of ? __ldg(a.slot_of + view) : view) : 0u;
                if (((sel >> (ub + vv)) & 1u) && rr < nrows && RLFC_DBG_INDEX_OK(a.dbg, ov, a.n_out)) {
                    uint8_t *dst = out_px<kPacked>(a, ov, by * 4 + rr, bx0 * 4) + k * unit;
                    const uint8_t *src = bb + (vv * 4 + rr) * (kNL * 4 * BPP) + k * unit;
                    if (unit == 4)
                        *reinterpret_cast<uint32_t *>(dst) = *reinterpret_cast<const uint32_t *>(src);
                    else
                        *dst = *src;
                }
            }
        }
        __syncwarp();
    }
}

template <bool kPacked>
int launch_decode(const rlfc_stream *s, uint8_t *d_out, const uint8_t *needed, const uint32_t *slot_of, uint32_t n_out,
                  cudaStream_t st)
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
        a.vec4 = ((uintptr_t)d_out & 3u) == 0;
    } else {
        a.vec16 = ((uintptr_t)d_out & 15u) == 0 && (a.W & 15u) == 0;
        a.vec4 = ((uintptr_t)d_out & 3u) == 0 && (a.W & 3u) == 0;
    }
    a.pmax = std::max<uint32_t>(s->max_strip_present, 1);
    a.n_units = (t.S + kUnit - 1) / kUnit;
    a.node_smem = t.S <= kNodeSmemMax;
    a.dbg = s->d_debug;
    a.n_out = n_out;
    a.ahead = 0;
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
    {
        int sms = 0, per_sm = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device) == cudaSuccess &&
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem) == cudaSuccess)
            a.ahead = (uint32_t)(std::max(sms, 0) * std::max(per_sm, 0));
    }
    { rlfc::TraceScope trace_((kPacked ? "decode_all_kernel<packed>" : "decode_all_kernel"), st); kern<<<grid, kThreads, smem, st>>>(a); }
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_fail(e, "decode_all launch");
    return RLFC_OK;
}

}  // namespace

int launch_decode_all(const rlfc_stream *s, uint8_t *d_out, cudaStream_t st)
{
    return launch_decode<false>(s, d_out, nullptr, nullptr, s->tab.n_views, st);
}

int launch_decode_packed(const rlfc_stream *s, uint32_t *d_out, const uint8_t *needed, const uint32_t *slot_of,
                         uint32_t n_slots, cudaStream_t st)
{
    return launch_decode<true>(s, reinterpret_cast<uint8_t *>(d_out), needed, slot_of, n_slots, st);
}

}  // namespace rlfc

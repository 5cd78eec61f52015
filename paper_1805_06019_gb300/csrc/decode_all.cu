// Full light-field decode: Algorithm 2 for every (view, block location).
//
// One CTA owns a strip of kNL consecutive block locations of one block row.
// Its 3 * kNL records (location-major, then Y / Co / Cg) and top-RKV blocks
// are read once.  Phases:
//  1. parse: one warp per record stores the presence mask, the stored-block
//     count in front of each mask word, and the payload bit offset of every
//     stored block (closed-form lengths of the 18-bit headers, warp scan);
//  2. internal nodes (levels >= 1, first in BFS order): their stored blocks
//     are decoded straight into the node's slab and the levels are added top
//     down, reconstruction = parent reconstruction (or top RKV) + residual;
//     then every parent of a view converts its reconstruction to RGB once;
//  3. the views, in batches of whole 16-position units whose stored blocks
//     fit kSlotCap decode slots:
//     a. one thread per (view, location) finds the blocks stored for it in
//        the three channel records; each such pair becomes an item with its
//        decode slots, each slot naming (record, rank);
//     b. every slot is decoded by one thread (a mode-generic BISE decoder:
//        the payload is aligned once, digits come from base-3 / base-5
//        tables, low parts from a per-thread column of the aligned bits);
//        meanwhile the batch's blocks are written as their parent's RGB,
//        which is the exact result for every block without a stored
//        residual (most of them);
//     c. every item (a block with at least one stored channel) adds its
//        residual rows to the parent rows, applies the inverse YCoCg-R two
//        pixels per instruction and overwrites its parent copy.
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
constexpr int kUnit = 16;                        // batch boundaries fall on multiples of 16 positions
constexpr int kSlotCap = 3 * kNL * kUnit;        // decode slots: any one unit fits
constexpr int kMaxUnits = 4;                     // units per batch at most
constexpr int kItemCap = kNL * kUnit * kMaxUnits;
constexpr int kCols = 6;                         // per-thread column words of the generic decoder
constexpr uint32_t kSmemBudget = 200 * 1024;

static_assert(kNL == 8, "the pair index split below assumes eight locations per strip");

// Reconstructions and residuals are held as 16-bit values plus a bias of
// 2^14, two to a word: then parent + residual is one 32-bit add for two
// values (no carry crosses a half while every value stays in
// [-2^14, 2^14)), and the inverse YCoCg-R runs on two pixels per
// instruction.
constexpr uint32_t kB2 = 0x40004000u;     // the bias in both halves (a zero pair)
constexpr uint32_t kHalfB2 = 0x20002000u;

__constant__ uint32_t c_modes[kNumModes] = RLFC_MODE_TABLE_INIT;

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
    uint32_t pmax;           // largest number of stored blocks in one record
    uint32_t n_units;        // ceil(S / kUnit)
};

// Words per block row of the parents' converted rows: 12 bytes RGB or four
// packed pixels.
template <bool kPacked>
__host__ __device__ constexpr uint32_t row_words() { return kPacked ? 4u : 3u; }

struct Smem {
    uint32_t *top;     // [n_top][kNL][24]  biased pairs
    uint32_t *inter;   // [n_int][kNL][24]  internal reconstructions, biased pairs
    uint32_t *prgb;    // [n_par][4][kNL][row_words]  parent rows converted to RGB
    uint32_t *mask;    // [kRecs][MW]
    uint32_t *mpre;    // [kRecs][MW]  stored blocks in front of each mask word
    uint32_t *need;    // [MW]  views to decode (bit per BFS position)
    uint16_t *ucnt;    // [n_units]  stored blocks of the views to decode, per unit of positions
    void *off;         // [kRecs][pmax]  payload bit offset of each stored block (OffT)
    uint32_t *slots;   // [kSlotCap][8]  decoded leaf blocks, biased pairs
    uint2 *sent;       // [kSlotCap]  (record | rank << 8, target word in inter or 0)
    uint32_t *items;   // [kItemCap]  p | l << 14 | stored channels << 18 | first slot << 21
    uint32_t *col;     // [kCols][kThreads]  generic decoder columns
};

extern __shared__ __align__(16) unsigned char g_smem[];

__host__ __device__ inline size_t r16(size_t b) { return (b + 15) & ~size_t(15); }

template <bool kPacked, typename OffT>
__device__ __forceinline__ Smem carve(const Args &a)
{
    Smem m;
    unsigned char *p = g_smem;
    m.slots = reinterpret_cast<uint32_t *>(p);
    p += r16(32ull * kSlotCap);
    m.top = reinterpret_cast<uint32_t *>(p);
    p += r16(96ull * a.n_top * kNL);
    m.inter = reinterpret_cast<uint32_t *>(p);
    p += r16(96ull * a.n_int * kNL);
    m.prgb = reinterpret_cast<uint32_t *>(p);
    p += r16(16ull * row_words<kPacked>() * a.n_par * kNL);
    m.mask = reinterpret_cast<uint32_t *>(p);
    p += r16(4ull * kRecs * a.MW);
    m.mpre = reinterpret_cast<uint32_t *>(p);
    p += r16(4ull * kRecs * a.MW);
    m.need = reinterpret_cast<uint32_t *>(p);
    p += r16(4ull * a.MW);
    m.sent = reinterpret_cast<uint2 *>(p);
    p += r16(8ull * kSlotCap);
    m.items = reinterpret_cast<uint32_t *>(p);
    p += r16(4ull * kItemCap);
    m.col = reinterpret_cast<uint32_t *>(p);
    p += r16(4ull * kCols * kThreads);
    m.ucnt = reinterpret_cast<uint16_t *>(p);
    p += r16(2ull * a.n_units);
    m.off = p;
    return m;
}

inline size_t smem_bytes(bool packed, uint32_t n_top, uint32_t n_int, uint32_t n_par, uint32_t MW, uint32_t n_units,
                         uint32_t pmax, size_t off_size)
{
    return r16(32ull * kSlotCap) + r16(96ull * n_top * kNL) + r16(96ull * n_int * kNL) +
           r16(16ull * (packed ? 4 : 3) * n_par * kNL) + 2 * r16(4ull * kRecs * MW) + r16(4ull * MW) +
           r16(8ull * kSlotCap) + r16(4ull * kItemCap) + r16(4ull * kCols * kThreads) + r16(2ull * n_units) +
           r16(off_size * kRecs * pmax);
}

// ---- one BISE block, any mode ---------------------------------------------
//
// The payload (at most 160 bits) is aligned to its first bit once, into
// seven words.  The digit words of a trit or quint block sit at fixed
// positions: their digits come from s_dig (base-3 digits of t < 256 at bits
// 3e, then base-5 digits of t < 128) and are gathered into one 64-bit word,
// digit v at bits 3v.  The low parts, at D + v * b for a b known only at run
// time, are read from the thread's column of the aligned bits in shared
// memory (column word k of thread t at k * kThreads + t: no bank conflicts).
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
            raw[k] = __ldg(w + k);
#pragma unroll
        for (int k = 0; k < 7; k++)
            A[k] = __funnelshift_r(raw[k], raw[k + 1], sh);
    }
    uint64_t dw = 0;
    uint32_t Lw[kCols];
    if (kind == 1) {
        // trits: three 8-bit digit words and a 2-bit one (values 15), then the low parts at bit 26
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
        col[k * kThreads] = Lw[k];
    const uint32_t lmask = (1u << b) - 1u;
    const uint32_t sb = scale << b;
    uint32_t u[kVals];
    uint32_t p = 0;
#pragma unroll
    for (int v = 0; v < kVals; v++) {
        const uint32_t k = p >> 5;
        const uint32_t lo = __funnelshift_r(col[k * kThreads], col[(k + 1) * kThreads], p & 31u) & lmask;
        const uint32_t d = (uint32_t)(dw >> (3 * v)) & 7u;
        u[v] = d * sb + lo * scale + base;
        p += b;
    }
#pragma unroll
    for (int j = 0; j < 8; j++)
        out[j] = __byte_perm(u[2 * j], u[2 * j + 1], 0x5410);
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

// Store one location's block row (four pixels from x) of view slot ov, row y.
template <bool kPacked>
__device__ __forceinline__ void store_row(const Args &a, uint32_t ov, uint32_t y, uint32_t x, const uint32_t w[4])
{
    const size_t px = ((size_t)ov * a.H + y) * a.W + x;
    const bool whole = x + 4 <= a.W;
    if (kPacked) {
        uint32_t *dst = reinterpret_cast<uint32_t *>(a.out) + px;
        if (whole && a.vec16) {
            *reinterpret_cast<uint4 *>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
        } else {
            for (uint32_t k = 0; k < 4 && x + k < a.W; k++)
                dst[k] = w[k];
        }
    } else {
        uint8_t *dst = a.out + px * 3;
        if (whole && a.vec4) {
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

// Output slot of a view: the table's entry (packed decode of the needed
// views) or the view itself.
__device__ __forceinline__ uint32_t out_slot(const Args &a, uint32_t view)
{
    return a.slot_of ? __ldg(a.slot_of + view) : view;
}

template <bool kPacked, typename OffT>
__global__ void __launch_bounds__(kThreads, 3) decode_all_kernel(const Args a)
{
    __shared__ uint32_t s_mode[32];   // modes >= 28 never pass the loader; their entries are 0
    __shared__ uint16_t s_dig[256 + 128];
    __shared__ uint32_t s_roff[kRecs];
    __shared__ uint32_t s_cnt[2][2];   // [batch parity] items, slots
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t bx0 = blockIdx.x * kNL, by = blockIdx.y;
    const uint32_t nl = min((uint32_t)kNL, a.nlx - bx0);
    const uint32_t b0 = by * a.nlx + bx0;
    const Smem m = carve<kPacked, OffT>(a);
    OffT *m_off = reinterpret_cast<OffT *>(m.off);
    constexpr uint32_t RW = row_words<kPacked>();

    // ---- set-up: tables, the strip's top-RKV blocks, zero reconstructions
    if (tid < 32)
        s_mode[tid] = tid < kNumModes ? c_modes[tid] : 0u;
    for (uint32_t t = tid; t < 256 + 128; t += kThreads) {
        // digits of t in base 3 (t < 256) or of t - 256 in base 5, three bits each
        const uint32_t base = t < 256 ? 3u : 5u, n = t < 256 ? 5u : 3u;
        uint32_t x = t < 256 ? t : t - 256, e = 0;
        for (uint32_t k = 0; k < n; k++) {
            e |= (x % base) << (3 * k);
            x /= base;
        }
        s_dig[t] = (uint16_t)e;
    }
    if (tid < kRecs)
        s_roff[tid] = tid < 3 * (int)nl ? __ldg(a.offsets + 3 * b0 + tid) : 0u;
    if (tid < 4)
        s_cnt[tid >> 1][tid & 1] = 0;
    {
        const uint32_t *tg = reinterpret_cast<const uint32_t *>(a.top);
        for (uint32_t i = tid; i < a.n_top * kNL * 24; i += kThreads) {
            const uint32_t t = i / (kNL * 24), rest = i - t * (kNL * 24), loc = rest / 24, wi = rest - loc * 24;
            m.top[i] = loc < nl ? (__ldg(tg + ((size_t)t * a.nloc + b0 + loc) * 24 + wi) ^ 0x80008000u) - kB2 : kB2;
        }
    }
    for (uint32_t i = tid; i < a.n_int * kNL * 24; i += kThreads)
        m.inter[i] = kB2;
    // the views to decode, one bit per BFS position (internal positions 0)
    for (uint32_t w0 = warp * 32; w0 < a.MW * 32; w0 += kWarps * 32) {
        const uint32_t p = w0 + lane;
        bool need = p >= a.n_int && p < a.S;
        if (need && kPacked && a.needed)
            need = __ldg(a.needed + node_view(__ldg(a.node_info + p))) != 0;
        const unsigned bal = __ballot_sync(kFullMask, need);
        if (lane == 0)
            m.need[w0 >> 5] = bal;
    }
    __syncthreads();   // the mode table and the record offsets are read below

    // ---- phase 1: per record, the payload offset of every stored block
    const uint32_t hdr0 = 32 * a.MW;
    for (uint32_t r = warp; r < kRecs; r += kWarps) {
        uint32_t *mk = m.mask + r * a.MW;
        uint32_t *mp = m.mpre + r * a.MW;
        if (r >= 3 * nl) {
            for (uint32_t w = lane; w < a.MW; w += 32) {
                mk[w] = 0;
                mp[w] = 0;
            }
            continue;
        }
        const uint32_t *rec = a.records + __ldg(a.offsets + 3 * b0 + r);
        uint32_t P = 0;
        for (uint32_t w0 = 0; w0 < a.MW; w0 += 32) {
            const uint32_t word = w0 + lane < a.MW ? __ldg(rec + w0 + lane) : 0u;
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
                const uint32_t mode = __funnelshift_r(__ldg(rec + (bp >> 5)), __ldg(rec + (bp >> 5) + 1), bp & 31u) & 31u;
                len = mode_bits(s_mode[mode]);
            }
            const uint32_t incl = warp_inclusive_scan(len, lane);
            if (h < P)
                m_off[r * a.pmax + h] = (OffT)(run + incl - len);
            run += __shfl_sync(kFullMask, incl, 31);
        }
    }
    __syncthreads();

    // stored blocks of the views to decode, per unit of kUnit positions
    for (uint32_t u = tid; u < a.n_units; u += kThreads) {
        const uint32_t w = u >> 1, sh = 16u * (u & 1u);
        const uint32_t nb = (m.need[w] >> sh) & 0xFFFFu;
        uint32_t c = 0;
        for (uint32_t r = 0; r < kRecs; r++)
            c += __popc((m.mask[r * a.MW + w] >> sh) & nb);
        m.ucnt[u] = (uint16_t)c;
    }

    // ---- phase 2: internal nodes.  Their stored blocks are decoded straight
    // into the node slabs, kSlotCap (node, record) pairs at a time.
    uint32_t *my_col = m.col + tid;
    const uint32_t n_pairs_int = a.n_int * kRecs;
    for (uint32_t i0 = 0; i0 < n_pairs_int; i0 += kSlotCap) {
        __syncthreads();
        const uint32_t i1 = min(n_pairs_int, i0 + kSlotCap);
        for (uint32_t ib = i0; ib < i1; ib += kThreads) {
            const uint32_t i = ib + tid;
            bool present = false;
            uint32_t r = 0, rank = 0, p = 0;
            if (i < i1) {
                p = i / kRecs;
                r = i - p * kRecs;
                const uint32_t word = m.mask[r * a.MW + (p >> 5)];
                present = (word >> (p & 31u)) & 1u;
                rank = m.mpre[r * a.MW + (p >> 5)] + __popc(word & ((1u << (p & 31u)) - 1u));
            }
            const unsigned bal = __ballot_sync(kFullMask, present);
            uint32_t at = 0;
            if (lane == 0 && bal)
                at = atomicAdd(&s_cnt[0][1], (uint32_t)__popc(bal));
            at = __shfl_sync(kFullMask, at, 0) + __popc(bal & ((1u << lane) - 1u));
            if (present) {
                const uint32_t loc = r / 3, c = r - 3 * loc;
                m.sent[at] = make_uint2(r | (rank << 8), (p * kNL + loc) * 24 + c * 8);
            }
        }
        __syncthreads();
        const uint32_t ns = s_cnt[0][1];
        for (uint32_t t = tid; t < ns; t += kThreads) {
            const uint2 e = m.sent[t];
            const uint32_t r = e.x & 255u, rank = e.x >> 8;
            const uint32_t *rec = a.records + s_roff[r];
            const uint32_t bp = hdr0 + kHdrBits * rank;
            const uint32_t hdr =
                __funnelshift_r(__ldg(rec + (bp >> 5)), __ldg(rec + (bp >> 5) + 1), bp & 31u) & 0x3FFFFu;
            uint32_t v[8];
            decode_block_generic(rec, m_off[r * a.pmax + rank], hdr, a.q, s_mode, s_dig, my_col, v);
            uint4 *d = reinterpret_cast<uint4 *>(m.inter + e.y);
            d[0] = make_uint4(v[0], v[1], v[2], v[3]);
            d[1] = make_uint4(v[4], v[5], v[6], v[7]);
        }
        __syncthreads();
        if (tid == 0)
            s_cnt[0][1] = 0;
    }
    __syncthreads();
    // levels top down: reconstruction = parent reconstruction + residual
    for (uint32_t g0 = 0; g0 < a.n_int;) {
        const uint32_t lvl = node_level(__ldg(a.node_info + g0));
        uint32_t g1 = g0 + 1;
        while (g1 < a.n_int && node_level(__ldg(a.node_info + g1)) == lvl)
            g1++;
        const uint32_t *src = lvl + 2 == a.L ? m.top : m.inter;
        for (uint32_t i = tid; i < (g1 - g0) * kNL * 6; i += kThreads) {
            const uint32_t p = g0 + i / (kNL * 6), rest = i % (kNL * 6);
            const uint4 s4 = reinterpret_cast<const uint4 *>(src)[node_parent(__ldg(a.node_info + p)) * (kNL * 6) + rest];
            uint4 &d4 = reinterpret_cast<uint4 *>(m.inter)[p * (kNL * 6) + rest];
            uint4 x = d4;
            x.x = x.x + s4.x - kB2;
            x.y = x.y + s4.y - kB2;
            x.z = x.z + s4.z - kB2;
            x.w = x.w + s4.w - kB2;
            d4 = x;
        }
        __syncthreads();
        g0 = g1;
    }
    // every parent of a view: its block rows as RGB, once per strip
    {
        const uint32_t *src = a.L == 2 ? m.top : m.inter;
        for (uint32_t i = tid; i < a.n_par * 4 * kNL; i += kThreads) {
            const uint32_t n = i / (4 * kNL), rest = i - n * (4 * kNL), rr = rest / kNL, l = rest - rr * kNL;
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

    // ---- phase 3: the views, in batches of whole units
    const uint32_t *par_slab = a.L == 2 ? m.top : m.inter;
    uint32_t parity = 0;
    for (uint32_t u0 = a.n_int / kUnit; u0 < a.n_units;) {
        // batch [P0, P1): units while their stored blocks fit the slots
        uint32_t k = 1, sum = m.ucnt[u0];
        while (k < kMaxUnits && u0 + k < a.n_units && sum + m.ucnt[u0 + k] <= (uint32_t)kSlotCap) {
            sum += m.ucnt[u0 + k];
            k++;
        }
        const uint32_t P0 = max(u0 * kUnit, a.n_int), P1 = min((u0 + k) * kUnit, a.S);
        u0 += k;
        uint32_t *cnt = s_cnt[parity];
        // (a) items: one thread per (position, location)
        const uint32_t npairs = (P1 - P0) * kNL;
        for (uint32_t ib = 0; ib < npairs; ib += kThreads) {
            const uint32_t i = ib + tid;
            uint32_t p = 0, l = 0, st3 = 0, w = 0, bit = 0;
            if (i < npairs) {
                p = P0 + (i >> 3);
                l = i & 7u;
                w = p >> 5;
                bit = p & 31u;
                if (l < nl && ((m.need[w] >> bit) & 1u)) {
#pragma unroll
                    for (uint32_t c = 0; c < 3; c++)
                        st3 |= ((m.mask[(3 * l + c) * a.MW + w] >> bit) & 1u) << c;
                }
            }
            const uint32_t n = (uint32_t)__popc(st3);
            const uint32_t incl = warp_inclusive_scan(n, lane);
            const unsigned bal = __ballot_sync(kFullMask, n != 0);
            uint32_t ibase = 0, sbase = 0;
            if (lane == 31 && bal) {
                ibase = atomicAdd(&cnt[0], (uint32_t)__popc(bal));
                sbase = atomicAdd(&cnt[1], incl);
            }
            ibase = __shfl_sync(kFullMask, ibase, 31);
            sbase = __shfl_sync(kFullMask, sbase, 31);
            if (n) {
                uint32_t slot = sbase + incl - n;
                m.items[ibase + __popc(bal & ((1u << lane) - 1u))] = p | (l << 14) | (st3 << 18) | (slot << 21);
#pragma unroll
                for (uint32_t c = 0; c < 3; c++) {
                    if ((st3 >> c) & 1u) {
                        const uint32_t r = 3 * l + c;
                        const uint32_t rank =
                            m.mpre[r * a.MW + w] + __popc(m.mask[r * a.MW + w] & ((1u << bit) - 1u));
                        m.sent[slot++] = make_uint2(r | (rank << 8), 0u);
                    }
                }
            }
        }
        __syncthreads();
        // (b) decode every slot; write every block of the batch as its parent's RGB
        {
            const uint32_t ns = cnt[1];
            for (uint32_t t = tid; t < ns; t += kThreads) {
                const uint32_t e = m.sent[t].x;
                const uint32_t r = e & 255u, rank = e >> 8;
                const uint32_t *rec = a.records + s_roff[r];
                const uint32_t bp = hdr0 + kHdrBits * rank;
                const uint32_t hdr =
                    __funnelshift_r(__ldg(rec + (bp >> 5)), __ldg(rec + (bp >> 5) + 1), bp & 31u) & 0x3FFFFu;
                uint32_t v[8];
                decode_block_generic(rec, m_off[r * a.pmax + rank], hdr, a.q, s_mode, s_dig, my_col, v);
                uint4 *d = reinterpret_cast<uint4 *>(m.slots + t * 8);
                d[0] = make_uint4(v[0], v[1], v[2], v[3]);
                d[1] = make_uint4(v[4], v[5], v[6], v[7]);
            }
            if (tid == 0) {
                s_cnt[parity ^ 1][0] = 0;
                s_cnt[parity ^ 1][1] = 0;
            }
            // copies: one thread per (position, block row, group of four locations)
            for (uint32_t i = tid; i < (P1 - P0) * 8; i += kThreads) {
                const uint32_t p = P0 + (i >> 3), rr = (i >> 1) & 3u, g = i & 1u;
                const uint32_t y = by * 4 + rr, l0 = 4 * g;
                if (!((m.need[p >> 5] >> (p & 31u)) & 1u) || y >= a.H || l0 >= nl)
                    continue;
                const uint32_t info = __ldg(a.node_info + p);
                const uint32_t ov = out_slot(a, node_view(info));
                const uint32_t *src = m.prgb + (((node_parent(info) - a.par_base) * 4 + rr) * kNL + l0) * RW;
                const uint32_t x = (bx0 + l0) * 4;
                if (a.vec16 && l0 + 4 <= nl && x + 16 <= a.W) {
                    const size_t px = ((size_t)ov * a.H + y) * a.W + x;
                    const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
                    uint4 *d4 = reinterpret_cast<uint4 *>(kPacked ? a.out + px * 4 : a.out + px * 3);
#pragma unroll
                    for (uint32_t k = 0; k < RW; k++)
                        d4[k] = s4[k];
                } else {
                    for (uint32_t l = l0; l < min(l0 + 4, nl); l++) {
                        uint32_t w[4];
#pragma unroll
                        for (uint32_t k = 0; k < RW; k++)
                            w[k] = src[(l - l0) * RW + k];
                        store_row<kPacked>(a, ov, y, (bx0 + l) * 4, w);
                    }
                }
            }
        }
        __syncthreads();
        // (c) blocks with a stored residual: parent + residual -> RGB, one
        // thread per (item, block row)
        {
            const uint32_t nit = cnt[0];
            for (uint32_t i = tid; i < nit * 4; i += kThreads) {
                const uint32_t it = m.items[i >> 2], rr = i & 3u;
                const uint32_t p = it & 0x3FFFu, l = (it >> 14) & 15u, st3 = (it >> 18) & 7u, s0 = it >> 21;
                const uint32_t y = by * 4 + rr;
                if (y >= a.H)
                    continue;
                const uint32_t info = __ldg(a.node_info + p);
                const uint32_t *ps = par_slab + (node_parent(info) * kNL + l) * 24 + rr * 2;
                uint2 ycc[3];
                uint32_t s = s0;
#pragma unroll
                for (uint32_t c = 0; c < 3; c++) {
                    const uint2 pb = *reinterpret_cast<const uint2 *>(ps + c * 8);
                    uint2 rb = make_uint2(kB2, kB2);
                    if ((st3 >> c) & 1u)
                        rb = *reinterpret_cast<const uint2 *>(m.slots + (s++) * 8 + rr * 2);
                    ycc[c] = make_uint2(pb.x + rb.x - kB2, pb.y + rb.y - kB2);
                }
                uint32_t w[4];
                row_to_rgb<kPacked>(ycc[0], ycc[1], ycc[2], w);
                store_row<kPacked>(a, out_slot(a, node_view(info)), y, (bx0 + l) * 4, w);
            }
        }
        __syncthreads();
        parity ^= 1;
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
    } else {
        a.vec16 = ((uintptr_t)d_out & 15u) == 0 && (a.W & 15u) == 0;
        a.vec4 = ((uintptr_t)d_out & 3u) == 0 && (a.W & 3u) == 0;
    }
    a.pmax = std::max<uint32_t>(s->max_present, 1);
    a.n_units = (t.S + kUnit - 1) / kUnit;
    // payload offsets are bit positions inside one record: 16 bits suffice
    // unless a record reaches 2^16 bits
    const bool off16 = (uint64_t)s->max_record_words * 32 < 65536;
    const size_t smem = smem_bytes(kPacked, a.n_top, a.n_int, a.n_par, a.MW, a.n_units, a.pmax, off16 ? 2 : 4);
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

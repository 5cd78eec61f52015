// Full light-field decode: Algorithm 2 for every (view, block location).
//
// One CTA owns a strip of kStrip consecutive block locations of one block
// row; their 3 * kStrip records (location-major, then Y / Co / Cg) and
// top-RKV blocks are read once (the records staged in shared memory when they
// fit).  Phases:
//  1. scan: one warp per record counts the stored blocks (popcounts of the
//     presence mask) and turns the closed-form payload lengths of their
//     headers into payload offsets with a warp scan;
//  2. internal nodes (levels >= 1, first in BFS order): their stored blocks
//     are compacted into a work list with their headers and sorted by BISE
//     mode, so that a warp decodes 32 blocks of one mode with that mode's
//     straight-line decoder (one thread per block); the levels are then added
//     top-down: reconstruction = parent reconstruction (or top RKV) +
//     residual;
//  3. the views (leaves), as many at a time (up to kLeafMax) as have at most
//     kResCap stored blocks over the strip: listed, sorted and decoded the
//     same way into compact slots (a per-(view, record) map points at them;
//     absent blocks read a slot of zeros), then parent + residual goes
//     through the inverse YCoCg-R two pixels at a time and each lane writes
//     its four pixels straight to the output row.
// Reconstructions are 16-bit values plus a bias of 2^14, two to a word (the
// loader refuses streams whose values could leave that range).  Every stored
// block of the strip is decoded once and every output byte is written once.
//
// A second instantiation writes one packed RGB word per pixel (r | g << 8 |
// b << 16) and decodes only the views a per-view mask asks for (its leaf
// batches run over the needed views alone); the renderer uses it to decode,
// from the compressed stream, just the views a batch of new cameras samples.
#include <cuda_runtime.h>

#include <algorithm>

#include "warp_decode.cuh"

namespace rlfc {
namespace {

constexpr int kStrip = (int)kDecodeStrip;   // block locations per CTA
constexpr uint32_t kStageCapWords = 8192;     // strip records staged in shared memory at most
constexpr size_t kCtaSmemTarget = 54 * 1024;  // dynamic shared memory per CTA that staging may fill up to
                                              // (four CTAs, static shared memory and the reserve fit an SM)
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kLeafMax = 64;      // views per leaf batch at most
constexpr int kResCap = 384;      // stored leaf blocks decoded per batch at most
constexpr uint32_t kZeroSlot = kResCap;   // a slot of zero residuals, for absent blocks
constexpr int kRecs = 3 * kStrip;
constexpr int kLS = 56;                 // int16 per location in a node slab (48 used; 28 words keep
                                        // a half-warp's 8-byte reads on distinct banks)
constexpr int kSlab = kStrip * kLS;     // int16 per node: [location][channel * 16 + value]
constexpr uint32_t kSmemBudget = 200 * 1024;

// Reconstructions and residuals are held as 16-bit values plus a bias of
// 2^14, two to a word: then parent + residual is one 32-bit add for two
// values (no carry crosses a half while every value stays in
// [-2^14, 2^14)), and the inverse YCoCg-R runs on two pixels per
// instruction.  The loader rejects streams whose values could leave that
// range.
constexpr uint32_t kB2 = 0x40004000u;     // the bias in both halves (a zero pair)
constexpr uint32_t kHalfB2 = 0x20002000u;

constexpr uint32_t kModeTable[kNumModes] = RLFC_MODE_TABLE_INIT;   // for the per-mode decoders
__constant__ uint32_t c_modes[kNumModes] = RLFC_MODE_TABLE_INIT;

struct Args {
    const uint32_t *records;
    const uint32_t *offsets;
    const int16_t *top;
    const uint32_t *node_info;
    uint8_t *out;          // RGB bytes, or packed RGB words (packed instantiation)
    const uint8_t *needed; // packed instantiation: per-view mask (nonzero = decode), may be null
    const uint32_t *slot_of; // packed instantiation with a mask: output slot of each needed view
    uint32_t S, n_int, n_top, L, q, MW;
    uint32_t nlx, nloc, W, H;
    uint32_t out_aligned16; // output base is 16-byte aligned
    uint32_t out_aligned4;  // output base is 4-byte aligned
    uint32_t pmax;          // largest number of stored blocks in one record
    uint32_t list_cap;      // work-list capacity (items)
    uint32_t stage_words;   // shared-memory words for the strip's records (0: read them from global)
};

struct Smem {
    uint32_t *node;    // [S]
    int16_t *top;      // [n_top][kSlab]  biased
    int16_t *inter;    // [n_int][kSlab]  internal reconstructions, biased
    int16_t *res;      // [kResCap + 1][16]  decoded leaf blocks, biased; also the unsorted work list
    uint16_t *map;     // [kLeafMax][kRecs]  slot of (leaf, record), kZeroSlot = not stored
    uint16_t *leafcnt; // [S - n_int]  stored blocks of each leaf (in batch order) over the strip
    uint16_t *leaves;  // [S - n_int]  with a view mask: the needed leaves, the order batches take
    uint32_t *mask;    // [kRecs][MW]
    uint32_t *mpre;    // [kRecs][MW]  stored blocks in front of each mask word
    void *off;         // [kRecs][pmax]  payload bit offset of each stored block (OffT)
    uint2 *list;       // [list_cap]  (node | record << 16, rank | header << 14), sorted by mode
    uint32_t *stage;   // [stage_words]  the strip's records, from a 16-byte boundary
};

extern __shared__ __align__(16) unsigned char g_smem[];

__host__ __device__ inline size_t r16(size_t b) { return (b + 15) & ~size_t(15); }

// The residual slots double as the unsorted work list.
__host__ __device__ inline size_t res_bytes(uint32_t list_cap)
{
    const size_t a = 32ull * (kResCap + 1), b = 8ull * list_cap;
    return r16(a > b ? a : b);
}

template <typename OffT>
__device__ __forceinline__ Smem carve(const Args &a)
{
    Smem m;
    unsigned char *p = g_smem;
    m.node = reinterpret_cast<uint32_t *>(p);
    p += r16(4ull * a.S);
    m.top = reinterpret_cast<int16_t *>(p);
    p += r16(2ull * a.n_top * kSlab);
    m.inter = reinterpret_cast<int16_t *>(p);
    p += r16(2ull * a.n_int * kSlab);
    m.res = reinterpret_cast<int16_t *>(p);
    p += res_bytes(a.list_cap);
    m.map = reinterpret_cast<uint16_t *>(p);
    p += r16(2ull * kLeafMax * kRecs);
    m.leafcnt = reinterpret_cast<uint16_t *>(p);
    p += r16(2ull * a.S);
    m.leaves = reinterpret_cast<uint16_t *>(p);
    p += r16(2ull * a.S);
    m.mask = reinterpret_cast<uint32_t *>(p);
    p += r16(4ull * kRecs * a.MW);
    m.mpre = reinterpret_cast<uint32_t *>(p);
    p += r16(4ull * kRecs * a.MW);
    m.off = p;
    p += r16(sizeof(OffT) * kRecs * a.pmax);
    m.list = reinterpret_cast<uint2 *>(p);
    p += r16(8ull * a.list_cap);
    m.stage = reinterpret_cast<uint32_t *>(p);
    return m;
}

inline size_t smem_bytes(uint32_t S, uint32_t n_top, uint32_t n_int, uint32_t MW, uint32_t pmax, uint32_t list_cap,
                         size_t off_size, uint32_t stage_words)
{
    return r16(4ull * S) + r16(2ull * n_top * kSlab) + r16(2ull * n_int * kSlab) + res_bytes(list_cap) +
           r16(2ull * kLeafMax * kRecs) + 2 * r16(2ull * S) + r16(4ull * kRecs * MW) + r16(4ull * kRecs * MW) +
           r16(off_size * kRecs * pmax) + r16(8ull * list_cap) + 4ull * stage_words;
}

// Where record r of the strip starts: rec_base + rec_off[r] (the staged copy
// in shared memory, or the stream).
struct RecSrc {
    const uint32_t *base;
    const uint32_t *off;   // [kRecs]
};

// ---- one BISE block in a mode known at compile time --------------------
//
// The payload's words are aligned to its first bit once; every digit group
// and low-bit field then sits at a fixed position.  Digit groups are split by
// table: s_digit[t] holds the base-3 digits of t (t < 256) at bits 2e, and
// s_digit[256 + t] the base-5 digits of t (t < 128) at bits 3e.  The 16
// values come out dequantised and biased, two to a word.
template <uint32_t K>
__device__ __forceinline__ void decode_block_k(const uint32_t *w, uint32_t sh, uint32_t scale, uint32_t base,
                                               const uint16_t *s_digit, uint32_t out[8])
{
    constexpr uint32_t M = kModeTable[K];
    constexpr uint32_t kind = M >> 12, b = (M >> 8) & 15u, bits = M & 255u;
    constexpr uint32_t D = kind == 1 ? 26u : (kind == 2 ? 38u : 0u);   // digit bits in front of the low parts
    constexpr uint32_t NA = (bits + 31u) / 32u;                        // aligned payload words
    if constexpr (bits == 0) {
#pragma unroll
        for (int j = 0; j < 8; j++)
            out[j] = __byte_perm(base, base, 0x5410);
    } else {
        uint32_t A[NA + 1];
        {
            uint32_t raw[NA + 1];
#pragma unroll
            for (uint32_t i = 0; i <= NA; i++)
                raw[i] = w[i];
#pragma unroll
            for (uint32_t i = 0; i < NA; i++)
                A[i] = __funnelshift_r(raw[i], raw[i + 1], sh);
            A[NA] = 0u;
        }
        // bits [P, P + Wd) of the aligned payload (P, Wd constant after unrolling)
        auto field = [&](uint32_t P, uint32_t Wd) -> uint32_t {
            const uint32_t i = P >> 5, s = P & 31u;
            const uint32_t mask = (1u << Wd) - 1u;
            return (s + Wd <= 32u ? (A[i] >> s) : __funnelshift_r(A[i], A[i + 1], s)) & mask;
        };
        uint32_t dg[6];
        if constexpr (kind == 1) {
#pragma unroll
            for (uint32_t g = 0; g < 3; g++)
                dg[g] = s_digit[field(8u * g, 8u)];
            const uint32_t t = field(24u, 2u);
            dg[3] = t == 3u ? 0u : t;
        } else if constexpr (kind == 2) {
#pragma unroll
            for (uint32_t g = 0; g < 5; g++)
                dg[g] = s_digit[256u + field(7u * g, 7u)];
            const uint32_t t = field(35u, 3u);
            dg[5] = t >= 5u ? t - 5u : t;
        }
        uint32_t u[kVals];
#pragma unroll
        for (uint32_t v = 0; v < (uint32_t)kVals; v++) {
            uint32_t digit = 0;
            if constexpr (kind == 1)
                digit = v == 15u ? dg[3] : (dg[v / 5u] >> (2u * (v % 5u))) & 3u;
            else if constexpr (kind == 2)
                digit = v == 15u ? dg[5] : (dg[v / 3u] >> (3u * (v % 3u))) & 7u;
            uint32_t low = 0;
            if constexpr (b > 0)
                low = field(D + v * b, b);
            u[v] = (digit << b) + low;
        }
#pragma unroll
        for (int j = 0; j < 8; j++)
            out[j] = __byte_perm(u[2 * j] * scale + base, u[2 * j + 1] * scale + base, 0x5410);
    }
}

__device__ __forceinline__ void decode_block(uint32_t mode, const uint32_t *w, uint32_t sh, uint32_t scale,
                                          uint32_t base, const uint16_t *s_digit, uint32_t out[8])
{
    switch (mode) {
#define RLFC_DECODE_CASE(K)                                   \
    case K:                                                   \
        decode_block_k<K>(w, sh, scale, base, s_digit, out);  \
        break;
        RLFC_DECODE_CASE(0) RLFC_DECODE_CASE(1) RLFC_DECODE_CASE(2) RLFC_DECODE_CASE(3)
        RLFC_DECODE_CASE(4) RLFC_DECODE_CASE(5) RLFC_DECODE_CASE(6) RLFC_DECODE_CASE(7)
        RLFC_DECODE_CASE(8) RLFC_DECODE_CASE(9) RLFC_DECODE_CASE(10) RLFC_DECODE_CASE(11)
        RLFC_DECODE_CASE(12) RLFC_DECODE_CASE(13) RLFC_DECODE_CASE(14) RLFC_DECODE_CASE(15)
        RLFC_DECODE_CASE(16) RLFC_DECODE_CASE(17) RLFC_DECODE_CASE(18) RLFC_DECODE_CASE(19)
        RLFC_DECODE_CASE(20) RLFC_DECODE_CASE(21) RLFC_DECODE_CASE(22) RLFC_DECODE_CASE(23)
        RLFC_DECODE_CASE(24) RLFC_DECODE_CASE(25) RLFC_DECODE_CASE(26) RLFC_DECODE_CASE(27)
#undef RLFC_DECODE_CASE
    default:   // modes >= 28 never pass the loader
#pragma unroll
        for (int j = 0; j < 8; j++)
            out[j] = kB2;
    }
}

// Stored blocks of the nodes at positions [q0, q1) of a node sequence
// (seq[q], or base + q without a list) over the strip's records, sorted by
// BISE mode into m.list (so that a warp decodes blocks of one mode
// together): item (j | record << 16, rank | header << 14), j = q - q0.  With
// `leaf`, map[j * kRecs + r] receives the item's list position (its decode
// slot) or kZeroSlot.  Returns the item count.
__device__ __forceinline__ uint32_t build_sorted(const Args &a, const Smem &m, const RecSrc &rs, uint32_t q0,
                                                 uint32_t q1, const uint16_t *seq, uint32_t base, bool leaf,
                                                 uint32_t *s_hist, uint32_t *s_count)
{
    const int tid = threadIdx.x, lane = tid & 31;
    uint2 *tmp = reinterpret_cast<uint2 *>(m.res);
    if (tid < 32)
        s_hist[tid] = 0;
    if (tid == 0)
        *s_count = 0;
    __syncthreads();
    const uint32_t hdr0 = 32 * a.MW;
    const uint32_t pairs = (q1 - q0) * kRecs;
    for (uint32_t i0 = 0; i0 < pairs; i0 += kThreads) {
        const uint32_t i = i0 + tid;
        bool present = false;
        uint32_t j = 0, r = 0, rank = 0, hdr = 0;
        if (i < pairs) {
            j = i / kRecs;
            r = i % kRecs;
            const uint32_t p = seq ? seq[q0 + j] : base + q0 + j;
            const uint32_t word = m.mask[r * a.MW + (p >> 5)];
            present = (word >> (p & 31u)) & 1u;
            if (present) {
                rank = m.mpre[r * a.MW + (p >> 5)] + __popc(word & ((1u << (p & 31u)) - 1u));
                hdr = get_bits(rs.base + rs.off[r], hdr0 + kHdrBits * rank, kHdrBits);
            }
            if (leaf && !present)
                m.map[i] = (uint16_t)kZeroSlot;
        }
        const unsigned bal = __ballot_sync(kFullMask, present);
        uint32_t at = 0;
        if (lane == 0 && bal)
            at = atomicAdd(s_count, (uint32_t)__popc(bal));
        at = __shfl_sync(kFullMask, at, 0) + __popc(bal & ((1u << lane) - 1u));
        const uint32_t mode = present ? hdr & 31u : 32u;
        const unsigned peers = __match_any_sync(kFullMask, mode);
        if (present) {
            tmp[at] = make_uint2(j | (r << 16), rank | (hdr << 14));
            if (lane == __ffs(peers) - 1)
                atomicAdd(&s_hist[mode], (uint32_t)__popc(peers));
        }
    }
    __syncthreads();
    if (tid < 32) {
        const uint32_t h = s_hist[tid];
        s_hist[tid] = warp_inclusive_scan(h, lane) - h;   // first position of each mode
    }
    __syncthreads();
    const uint32_t count = *s_count;
    for (uint32_t i0 = 0; i0 < count; i0 += kThreads) {
        const uint32_t i = i0 + tid;
        uint2 it = make_uint2(0u, 0u);
        if (i < count)
            it = tmp[i];
        const uint32_t mode = i < count ? (it.y >> 14) & 31u : 32u;
        const unsigned peers = __match_any_sync(kFullMask, mode);
        const int leader = __ffs(peers) - 1;
        uint32_t at = 0;
        if (i < count && lane == leader)
            at = atomicAdd(&s_hist[mode], (uint32_t)__popc(peers));
        at = __shfl_sync(kFullMask, at, leader) + __popc(peers & ((1u << lane) - 1u));
        if (i < count) {
            m.list[at] = it;
            if (leaf)
                m.map[(it.x & 0xFFFFu) * kRecs + (it.x >> 16)] = (uint16_t)at;
        }
    }
    __syncthreads();
    return count;
}

// Decode the sorted list: internal blocks into their node's slab at
// (node, location, channel), leaf blocks into slot = list position.
template <typename OffT>
__device__ __forceinline__ void decode_sorted(const Args &a, const Smem &m, const uint16_t *s_digit, uint32_t count,
                                              const RecSrc &rs, bool leaf)
{
    const OffT *off = reinterpret_cast<const OffT *>(m.off);
    for (uint32_t i = threadIdx.x; i < count; i += kThreads) {
        const uint2 it = m.list[i];
        const uint32_t r = it.x >> 16, rank = it.y & 0x3FFFu, hdr = it.y >> 14;
        const uint32_t pos = off[r * a.pmax + rank];
        const int32_t mn = ((int32_t)(hdr << 14)) >> 21;   // header bits 7..17, sign-extended
        const uint32_t scale = 1u << (a.q + ((hdr >> 5) & 3u));
        const uint32_t base = (uint32_t)mn * scale + 0x4000u;
        uint32_t v[8];
        decode_block(hdr & 31u, rs.base + rs.off[r] + (pos >> 5), pos & 31u, scale, base, s_digit, v);
        int16_t *dst;
        if (leaf) {
            dst = m.res + (size_t)i * kVals;
        } else {
            const uint32_t p = it.x & 0xFFFFu, loc = r / 3, c = r - 3 * loc;   // internal pass: j = node
            dst = m.inter + p * kSlab + loc * kLS + c * 16;
        }
        uint4 *d = reinterpret_cast<uint4 *>(dst);
        d[0] = make_uint4(v[0], v[1], v[2], v[3]);
        d[1] = make_uint4(v[4], v[5], v[6], v[7]);
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

template <bool kPacked, typename OffT>
__global__ void __launch_bounds__(kThreads, 4) decode_all_kernel(const Args a)
{
    __shared__ uint32_t s_mode[kNumModes];
    __shared__ uint16_t s_digit[256 + 128];
    __shared__ uint32_t s_hist[32];
    __shared__ uint32_t s_count;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t bx0 = blockIdx.x * kStrip, by = blockIdx.y;
    const uint32_t nl = min((uint32_t)kStrip, a.nlx - bx0);
    const uint32_t b0 = by * a.nlx + bx0;
    const Smem m = carve<OffT>(a);
    OffT *m_off = reinterpret_cast<OffT *>(m.off);

    if (tid < kNumModes)
        s_mode[tid] = c_modes[tid];
    for (uint32_t t = tid; t < 256 + 128; t += kThreads) {
        // digits of t in base 3 (t < 256) or of t - 256 in base 5
        const uint32_t base = t < 256 ? 3u : 5u, width = t < 256 ? 2u : 3u, n = t < 256 ? 5u : 3u;
        uint32_t x = t < 256 ? t : t - 256, e = 0;
        for (uint32_t k = 0; k < n; k++) {
            e |= (x % base) << (width * k);
            x /= base;
        }
        s_digit[t] = (uint16_t)e;
    }
    for (uint32_t i = tid; i < a.S; i += kThreads)
        m.node[i] = a.node_info[i];
    {
        // top RKV blocks, biased, two values per word
        uint32_t *tw = reinterpret_cast<uint32_t *>(m.top);
        const uint32_t *tg = reinterpret_cast<const uint32_t *>(a.top);
        for (uint32_t i = tid; i < a.n_top * kStrip * 24; i += kThreads) {
            const uint32_t t = i / (kStrip * 24), rest = i - t * (kStrip * 24), loc = rest / 24, wi = rest - loc * 24;
            tw[t * (kSlab / 2) + loc * (kLS / 2) + wi] =
                loc < nl ? (tg[((size_t)t * a.nloc + b0 + loc) * 24 + wi] ^ 0x80008000u) - kB2 : kB2;
        }
    }
    for (uint32_t i = tid; i < a.n_int * kSlab / 2; i += kThreads)
        reinterpret_cast<uint32_t *>(m.inter)[i] = kB2;
    for (uint32_t i = tid; i < kVals / 2; i += kThreads)
        reinterpret_cast<uint32_t *>(m.res + kZeroSlot * kVals)[i] = kB2;
    // the strip's records are contiguous in the stream: stage them (from a
    // 16-byte boundary, plus the two words the bit reader may read past a
    // record; the stream ends in zero padding) when they fit
    __shared__ uint32_t s_roff[kRecs];
    const uint32_t w_lo = a.offsets[3 * b0] & ~3u;
    const uint32_t n4 = (a.offsets[3 * (b0 + nl)] + 2 - w_lo + 3) / 4;
    const bool staged = 4 * n4 <= a.stage_words;
    if (staged) {
        const uint4 *src = reinterpret_cast<const uint4 *>(a.records + w_lo);
        uint4 *dst = reinterpret_cast<uint4 *>(m.stage);
        for (uint32_t i = tid; i < n4; i += kThreads)
            dst[i] = src[i];
    }
    for (uint32_t r = tid; r < kRecs; r += kThreads)
        s_roff[r] = r < 3 * nl ? a.offsets[3 * b0 + r] - (staged ? w_lo : 0u) : 0u;
    const RecSrc rs{staged ? m.stage : a.records, s_roff};
    __syncthreads();

    // ---- phase 1: per record, the payload offset of every stored block
    const uint32_t hdr0 = 32 * a.MW;
    for (uint32_t r = warp; r < kRecs; r += kWarps) {
        const uint32_t loc = r / 3;
        uint32_t *mk = m.mask + r * a.MW;
        if (loc >= nl) {
            for (uint32_t w = lane; w < a.MW; w += 32)
                mk[w] = 0;
            continue;
        }
        const uint32_t *rec = rs.base + rs.off[r];
        uint32_t P = 0;
        for (uint32_t w0 = 0; w0 < a.MW; w0 += 32) {
            const uint32_t word = w0 + lane < a.MW ? rec[w0 + lane] : 0u;
            const uint32_t cnt = (uint32_t)__popc(word);
            const uint32_t incl = warp_inclusive_scan(cnt, lane);
            if (w0 + lane < a.MW) {
                mk[w0 + lane] = word;
                m.mpre[r * a.MW + w0 + lane] = P + incl - cnt;
            }
            P += __shfl_sync(kFullMask, incl, 31);
        }
        uint32_t run = hdr0 + kHdrBits * P;
        for (uint32_t h0 = 0; h0 < P; h0 += 32) {
            const uint32_t h = h0 + lane;
            const uint32_t len = h < P ? mode_bits(s_mode[get_bits(rec, hdr0 + kHdrBits * h, 5)]) : 0u;
            const uint32_t incl = warp_inclusive_scan(len, lane);
            if (h < P)
                m_off[r * a.pmax + h] = (OffT)(run + incl - len);
            run += __shfl_sync(kFullMask, incl, 31);
        }
    }
    __syncthreads();

    // ---- phases 2 and 3 share one loop (one copy of the list builder and of
    // the per-mode decoders): the first pass takes the internal nodes
    // (levels >= 1, first in BFS order), decodes them into their slabs and
    // reconstructs them level by level; every later pass takes a batch of up
    // to kLeafMax views whose stored blocks fit the kResCap decode slots
    const bool use_mask = kPacked && a.needed != nullptr;
    __shared__ uint32_t s_p1, s_nleaf;
    // the leaf sequence the batches take: every leaf in BFS order, or, with a
    // view mask, only the needed leaves (compacted)
    if (use_mask) {
        if (tid == 0)
            s_nleaf = 0;
        __syncthreads();
        for (uint32_t b = a.n_int; b < a.S; b += kThreads) {
            const uint32_t p = b + tid;
            const bool need = p < a.S && a.needed[node_view(m.node[p])] != 0;
            const unsigned bal = __ballot_sync(kFullMask, need);
            uint32_t at = 0;
            if (lane == 0 && bal)
                at = atomicAdd(&s_nleaf, (uint32_t)__popc(bal));
            at = __shfl_sync(kFullMask, at, 0) + __popc(bal & ((1u << lane) - 1u));
            if (need)
                m.leaves[at] = (uint16_t)p;
        }
        __syncthreads();
    }
    const uint32_t nleaf = use_mask ? s_nleaf : a.S - a.n_int;
    const uint16_t *seq = use_mask ? m.leaves : nullptr;
    auto leaf_node = [&](uint32_t q) -> uint32_t { return use_mask ? (uint32_t)m.leaves[q] : a.n_int + q; };
    // stored blocks of each leaf of the sequence over the strip, and the
    // zero slot (which the internal pass's unsorted list may have covered)
    auto prepare_leaves = [&]() {
        for (uint32_t i = tid; i < kVals / 2; i += kThreads)
            reinterpret_cast<uint32_t *>(m.res + kZeroSlot * kVals)[i] = kB2;
        for (uint32_t q = tid; q < nleaf; q += kThreads) {
            const uint32_t p = leaf_node(q);
            uint32_t c = 0;
            for (uint32_t r = 0; r < kRecs; r++)
                c += (m.mask[r * a.MW + (p >> 5)] >> (p & 31u)) & 1u;
            m.leafcnt[q] = (uint16_t)c;
        }
    };
    bool internal = a.n_int > 0;
    if (!internal)
        prepare_leaves();
    for (uint32_t q0 = 0; internal || q0 < nleaf;) {
        __syncthreads();
        if (internal) {
            if (tid == 0)
                s_p1 = a.n_int;
        } else if (warp == 0) {
            // the longest run of sequence positions from q0 whose stored blocks fit
            uint32_t sum = 0, q1 = q0;
            const uint32_t lim = min(nleaf, q0 + kLeafMax);
            for (uint32_t b = q0; b < lim; b += 32) {
                const uint32_t q = b + lane;
                const uint32_t c = q < lim ? m.leafcnt[q] : (uint32_t)kResCap + 1;
                const uint32_t incl = warp_inclusive_scan(c, lane);
                const unsigned ok = __ballot_sync(kFullMask, sum + incl <= (uint32_t)kResCap);
                const uint32_t n_ok = __popc(ok);
                if (n_ok)
                    sum += __shfl_sync(kFullMask, incl, n_ok - 1);
                q1 = b + n_ok;
                if (n_ok < 32)
                    break;
            }
            if (lane == 0)
                s_p1 = max(q1, q0 + 1);
        }
        __syncthreads();
        const uint32_t q1 = s_p1, nb = q1 - q0;
        // the internal pass takes nodes [0, n_int); a leaf batch positions
        // [q0, q1) of the leaf sequence
        const uint32_t cnt = build_sorted(a, m, rs, internal ? 0u : q0, q1, internal ? nullptr : seq,
                                          internal ? 0u : a.n_int, !internal, s_hist, &s_count);
        decode_sorted<OffT>(a, m, s_digit, cnt, rs, !internal);
        __syncthreads();
        if (internal) {
            for (uint32_t b0 = 0; b0 < a.n_int;) {
                const uint32_t lvl = node_level(m.node[b0]);
                uint32_t b1 = b0;
                while (b1 < a.n_int && node_level(m.node[b1]) == lvl)
                    b1++;
                const uint4 *src = reinterpret_cast<const uint4 *>(lvl + 2 == a.L ? m.top : m.inter);
                uint4 *dst = reinterpret_cast<uint4 *>(m.inter);
                constexpr uint32_t kQ = kSlab / 8;   // uint4 per node slab
                for (uint32_t i = tid; i < (b1 - b0) * kQ; i += kThreads) {
                    const uint32_t p = b0 + i / kQ, rest = i % kQ;
                    const uint4 s4 = src[node_parent(m.node[p]) * kQ + rest];
                    uint4 d4 = dst[p * kQ + rest];
                    d4.x = d4.x + s4.x - kB2;
                    d4.y = d4.y + s4.y - kB2;
                    d4.z = d4.z + s4.z - kB2;
                    d4.w = d4.w + s4.w - kB2;
                    dst[p * kQ + rest] = d4;
                }
                __syncthreads();
                b0 = b1;
            }
            prepare_leaves();
            internal = false;
            continue;
        }
        // parent + residual -> RGB: one view per warp step, lane = (block
        // row, location), four pixels per lane written straight to the
        // output row
        for (uint32_t j = warp; j < nb; j += kWarps) {
            const uint32_t info = m.node[leaf_node(q0 + j)];
            const uint32_t view = node_view(info);
            const uint32_t row = (uint32_t)lane / kStrip, loc = (uint32_t)lane % kStrip;
            const uint32_t y = by * 4 + row, x = (bx0 + loc) * 4;
            if (loc >= nl || y >= a.H)
                continue;
            const int16_t *par = (a.L == 2 ? m.top : m.inter) + node_parent(info) * kSlab + loc * kLS + row * 4;
            uint2 ycc[3];
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const uint2 pb = *reinterpret_cast<const uint2 *>(par + c * 16);
                const uint32_t slot = m.map[j * kRecs + loc * 3 + c];
                const uint2 rb = *reinterpret_cast<const uint2 *>(m.res + slot * kVals + row * 4);
                ycc[c] = make_uint2(pb.x + rb.x - kB2, pb.y + rb.y - kB2);
            }
            uint32_t r01, g01, b01, r23, g23, b23;
            ycocg_pair_to_rgb(ycc[0].x, ycc[1].x, ycc[2].x, r01, g01, b01);
            ycocg_pair_to_rgb(ycc[0].y, ycc[1].y, ycc[2].y, r23, g23, b23);
            const uint32_t t01 = __byte_perm(r01, g01, 0x6240);   // R0 G0 R1 G1
            const uint32_t t23 = __byte_perm(r23, g23, 0x6240);   // R2 G2 R3 G3
            const bool whole = x + 4 <= a.W;
            if (kPacked) {
                const uint32_t px[4] = {__byte_perm(t01, b01, 0x0410) & 0xFFFFFFu,
                                        __byte_perm(t01, b01, 0x0632) & 0xFFFFFFu,
                                        __byte_perm(t23, b23, 0x0410) & 0xFFFFFFu,
                                        __byte_perm(t23, b23, 0x0632) & 0xFFFFFFu};
                const uint32_t ov = a.slot_of ? a.slot_of[view] : view;
                uint32_t *dst = reinterpret_cast<uint32_t *>(a.out) + ((size_t)ov * a.H + y) * a.W + x;
                if (whole && a.out_aligned16 && (a.W & 3u) == 0) {
                    *reinterpret_cast<uint4 *>(dst) = make_uint4(px[0], px[1], px[2], px[3]);
                } else {
                    for (uint32_t k = 0; k < 4 && x + k < a.W; k++)
                        dst[k] = px[k];
                }
            } else {
                // 4 pixels = 12 bytes: R0 G0 B0 R1 | G1 B1 R2 G2 | B2 R3 G3 B3
                const uint32_t w0 = __byte_perm(t01, b01, 0x2410);
                const uint32_t w1 = __byte_perm(__byte_perm(t01, b01, 0x0063), t23, 0x5410);
                const uint32_t w2 = __byte_perm(b23, t23, 0x2760);
                uint8_t *dst = a.out + (((size_t)view * a.H + y) * a.W + x) * 3;
                if (whole && a.out_aligned4 && (a.W & 3u) == 0) {
                    uint32_t *d = reinterpret_cast<uint32_t *>(dst);
                    d[0] = w0;
                    d[1] = w1;
                    d[2] = w2;
                } else {
                    const uint32_t wv[3] = {w0, w1, w2};
                    for (uint32_t k = 0; k < 12 && x + k / 3 < a.W; k++)
                        dst[k] = (uint8_t)(wv[k >> 2] >> (8 * (k & 3)));
                }
            }
        }
        q0 = q1;
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
    a.out_aligned16 = ((uintptr_t)d_out & 15u) == 0;
    a.out_aligned4 = ((uintptr_t)d_out & 3u) == 0;
    a.pmax = std::max<uint32_t>(s->max_present, 1);
    a.list_cap = std::max<uint32_t>(kRecs * t.n_int, kResCap);
    // payload offsets are bit positions inside one record: 16 bits suffice
    // unless a record reaches 2^16 bits
    const bool off16 = (uint64_t)s->max_record_words * 32 < 65536;
    // staging for the largest strip's records (16-byte boundary, bit-reader
    // slack), within what keeps a CTA at kCtaSmemTarget bytes; strips whose
    // records do not fit read them from the stream
    const size_t base = smem_bytes(a.S, a.n_top, a.n_int, a.MW, a.pmax, a.list_cap, off16 ? 2 : 4, 0);
    const size_t room = base < kCtaSmemTarget ? (kCtaSmemTarget - base) / 4 : 0;
    a.stage_words = (uint32_t)std::min<size_t>({(size_t)((s->max_strip_words + 8 + 3) & ~3u),
                                                (size_t)kStageCapWords, room & ~size_t(3)});
    const size_t smem = base + 4ull * a.stage_words;
    if (smem > kSmemBudget || a.S >= 65536) {
        set_error("tree too large for the decode-all kernel's shared memory");
        return RLFC_E_UNSUPPORTED;
    }
    auto kern = off16 ? decode_all_kernel<kPacked, uint16_t> : decode_all_kernel<kPacked, uint32_t>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return cuda_fail(e, "decode_all: shared memory attribute");
    dim3 grid((a.nlx + kStrip - 1) / kStrip, s->info.nloc_y);
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

// Full light-field decode: Algorithm 2 for every (view, block location).
//
// One CTA owns a strip of kStrip consecutive block locations of one block
// row; their 3 * kStrip records (location-major, then Y / Co / Cg) and
// top-RKV blocks are read once.  Phases:
//  1. scan: one warp per record counts the stored blocks (popcounts of the
//     presence mask) and turns the closed-form payload lengths of their
//     headers into payload offsets with a warp scan;
//  2. internal nodes (levels >= 1, first in BFS order): the stored blocks are
//     compacted into a work list (no thread idles on an absent node) and each
//     thread decodes whole blocks with a sequential bit reader; the levels are
//     then added top-down: reconstruction = parent reconstruction (or top
//     RKV) + residual;
//  3. the views (leaves), as many at a time (up to kLeafMax) as have at most
//     kResCap stored blocks over the strip: compacted, decoded the same way
//     into compact slots (a per-(view, record) map points at them; absent
//     blocks add nothing), then parent + residual is converted from YCoCg-R
//     to RGB and written as whole image rows with 16-byte stores.
// Every stored block of the strip is decoded once and every output byte is
// written once.
//
// A second instantiation writes one packed RGB word per pixel (r | g << 8 |
// b << 16) and decodes only the views a per-view mask asks for; the renderer
// uses it to decode, from the compressed stream, just the views a batch of
// new cameras samples.
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
constexpr int kRecs = 3 * kStrip;
constexpr int kRowsPerJob = 32 / kStrip;   // block rows a warp converts per step (lane = row, location)
constexpr int kLS = 56;                 // int16 per location in a node slab (48 used; 28 words keep
                                        // a half-warp's 8-byte reads on distinct banks)
constexpr int kSlab = kStrip * kLS;     // int16 per node: [location][channel * 16 + value]
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
    uint32_t out_aligned4;  // output base is 4-byte aligned
    uint32_t pmax;          // largest number of stored blocks in one record
    uint32_t list_cap;      // work-list capacity (items)
    uint32_t stage_words;   // shared-memory words for the strip's records (0: read them from global)
};

struct Smem {
    uint32_t *node;    // [S]
    int16_t *top;      // [n_top][kSlab]
    int16_t *inter;    // [n_int][kSlab]  internal reconstructions
    int16_t *res;      // [kResCap][16]  decoded leaf blocks, one slot per listed block
    uint16_t *map;     // [kLeafMax][kRecs]  slot of (leaf, record), 0xFFFF = not stored
    uint16_t *leafcnt; // [S - n_int]  stored blocks of each leaf over the strip
    uint32_t *mask;    // [kRecs][MW]
    uint32_t *mpre;    // [kRecs][MW]  stored blocks in front of each mask word
    void *off;         // [kRecs][pmax]  payload bit offset of each stored block (OffT)
    uint2 *list;       // [list_cap]  (node | record << 16, rank)
    uint32_t *stage;   // [stage_words]  the strip's records, from a 16-byte boundary
};

extern __shared__ __align__(16) unsigned char g_smem[];

__host__ __device__ inline size_t r16(size_t b) { return (b + 15) & ~size_t(15); }

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
    p += r16(32ull * kResCap);
    m.map = reinterpret_cast<uint16_t *>(p);
    p += r16(2ull * kLeafMax * kRecs);
    m.leafcnt = reinterpret_cast<uint16_t *>(p);
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
    return r16(4ull * S) + r16(2ull * n_top * kSlab) + r16(2ull * n_int * kSlab) +
           r16(32ull * kResCap) + r16(2ull * kLeafMax * kRecs) + r16(2ull * S) +
           r16(4ull * kRecs * MW) + r16(4ull * kRecs * MW) + r16(off_size * kRecs * pmax) + r16(8ull * list_cap) +
           4ull * stage_words;
}

// Where record r of the strip starts: rec_base + rec_off[r] (the staged copy
// in shared memory, or the stream).
struct RecSrc {
    const uint32_t *base;
    const uint32_t *off;   // [kRecs]
};

// Stored blocks of nodes [p0, p1) over the strip's records, compacted into the
// work list: (node | record << 16, rank).  Returns the item count.
__device__ __forceinline__ uint32_t build_list(const Args &a, const Smem &m, uint32_t p0, uint32_t p1,
                                               uint32_t *s_count, bool use_mask)
{
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid == 0)
        *s_count = 0;
    __syncthreads();
    const uint32_t pairs = (p1 - p0) * kRecs;
    for (uint32_t i0 = 0; i0 < pairs; i0 += kThreads) {
        const uint32_t i = i0 + tid;
        bool present = false;
        uint32_t p = 0, r = 0, rank = 0;
        if (i < pairs) {
            p = p0 + i / kRecs;
            r = i % kRecs;
            const uint32_t word = m.mask[r * a.MW + (p >> 5)];
            present = (word >> (p & 31u)) & 1u;
            if (present && use_mask)
                present = a.needed[node_view(m.node[p])] != 0;
            if (present)
                rank = m.mpre[r * a.MW + (p >> 5)] + __popc(word & ((1u << (p & 31u)) - 1u));
        }
        const unsigned bal = __ballot_sync(kFullMask, present);
        uint32_t base = 0;
        if (lane == 0 && bal)
            base = atomicAdd(s_count, (uint32_t)__popc(bal));
        base = __shfl_sync(kFullMask, base, 0);
        if (present)
            m.list[base + __popc(bal & ((1u << lane) - 1u))] = make_uint2(p | (r << 16), rank);
    }
    __syncthreads();
    return *s_count;
}

// One listed block, one thread: the residual (min + u) * 2^(q + shift) of its
// 16 values, read with the sequential bit reader.
template <typename OffT>
__device__ __forceinline__ void decode_item(const Args &a, const Smem &m, const uint32_t *s_mode, uint2 it,
                                            const RecSrc &rs, int32_t val[kVals])
{
    const OffT *off = reinterpret_cast<const OffT *>(m.off);
    const uint32_t rank = it.y, r = it.x >> 16;
    const uint32_t *rec = rs.base + rs.off[r];
    const BlockHeader h = unpack_header(get_bits(rec, 32 * a.MW + kHdrBits * rank, kHdrBits));
    int32_t u[kVals];
    bise_decode16(rec, off[r * a.pmax + rank], s_mode[h.mode], u);
    const int32_t scale = 1 << (a.q + h.shift);
#pragma unroll
    for (int v = 0; v < kVals; v++)
        val[v] = (h.min + u[v]) * scale;
}

// Internal nodes: each listed block into its node's slab,
// dst[(node - p0) * kSlab + location * kLS + channel * 16 + value].
template <typename OffT>
__device__ __forceinline__ void decode_list(const Args &a, const Smem &m, const uint32_t *s_mode, uint32_t count,
                                            const RecSrc &rs, uint32_t p0, int16_t *dst)
{
    for (uint32_t i = threadIdx.x; i < count; i += kThreads) {
        const uint2 it = m.list[i];
        int32_t val[kVals];
        decode_item<OffT>(a, m, s_mode, it, rs, val);
        const uint32_t p = it.x & 0xFFFFu, r = it.x >> 16;
        const uint32_t loc = r / 3, c = r - 3 * loc;
        uint2 *d = reinterpret_cast<uint2 *>(dst + (p - p0) * kSlab + loc * kLS + c * 16);
#pragma unroll
        for (int v = 0; v < kVals; v += 4)
            d[v >> 2] = make_uint2(((uint32_t)val[v] & 0xFFFFu) | ((uint32_t)val[v + 1] << 16),
                                   ((uint32_t)val[v + 2] & 0xFFFFu) | ((uint32_t)val[v + 3] << 16));
    }
}

// Leaves: listed block i into compact slot i (16 int16, two 16-byte stores).
template <typename OffT>
__device__ __forceinline__ void decode_leaf_list(const Args &a, const Smem &m, const uint32_t *s_mode,
                                                 uint32_t count, const RecSrc &rs)
{
    for (uint32_t i = threadIdx.x; i < count; i += kThreads) {
        int32_t val[kVals];
        decode_item<OffT>(a, m, s_mode, m.list[i], rs, val);
        uint32_t w[8];
#pragma unroll
        for (int v = 0; v < kVals; v += 2)
            w[v >> 1] = ((uint32_t)val[v] & 0xFFFFu) | ((uint32_t)val[v + 1] << 16);
        uint4 *d = reinterpret_cast<uint4 *>(m.res + (size_t)i * kVals);
        d[0] = make_uint4(w[0], w[1], w[2], w[3]);
        d[1] = make_uint4(w[4], w[5], w[6], w[7]);
    }
}

// Stored blocks of leaves [p0, p1) over the strip's records, compacted into
// the work list (slot = list position); map[(p - p0) * kRecs + r] receives
// the slot of (leaf p, record r) or 0xFFFF.  Returns the item count.
__device__ __forceinline__ uint32_t build_leaf_list(const Args &a, const Smem &m, uint32_t p0, uint32_t p1,
                                                    uint32_t *s_count, bool use_mask)
{
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid == 0)
        *s_count = 0;
    __syncthreads();
    const uint32_t pairs = (p1 - p0) * kRecs;
    for (uint32_t i0 = 0; i0 < pairs; i0 += kThreads) {
        const uint32_t i = i0 + tid;
        bool present = false;
        uint32_t p = 0, r = 0, rank = 0;
        if (i < pairs) {
            p = p0 + i / kRecs;
            r = i % kRecs;
            const uint32_t word = m.mask[r * a.MW + (p >> 5)];
            present = (word >> (p & 31u)) & 1u;
            if (present && use_mask)
                present = a.needed[node_view(m.node[p])] != 0;
            if (present)
                rank = m.mpre[r * a.MW + (p >> 5)] + __popc(word & ((1u << (p & 31u)) - 1u));
        }
        const unsigned bal = __ballot_sync(kFullMask, present);
        uint32_t base = 0;
        if (lane == 0 && bal)
            base = atomicAdd(s_count, (uint32_t)__popc(bal));
        base = __shfl_sync(kFullMask, base, 0);
        const uint32_t slot = base + __popc(bal & ((1u << lane) - 1u));
        if (present)
            m.list[slot] = make_uint2(p | (r << 16), rank);
        if (i < pairs)
            m.map[i] = present ? (uint16_t)slot : (uint16_t)0xFFFFu;
    }
    __syncthreads();
    return *s_count;
}

template <bool kPacked, typename OffT>
__global__ void __launch_bounds__(kThreads, 4) decode_all_kernel(const Args a)
{
    __shared__ uint32_t s_mode[kNumModes];
    __shared__ uint32_t s_count;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t bx0 = blockIdx.x * kStrip, by = blockIdx.y;
    const uint32_t nl = min((uint32_t)kStrip, a.nlx - bx0);
    const uint32_t b0 = by * a.nlx + bx0;
    const Smem m = carve<OffT>(a);
    OffT *m_off = reinterpret_cast<OffT *>(m.off);

    if (tid < kNumModes)
        s_mode[tid] = c_modes[tid];
    for (uint32_t i = tid; i < a.S; i += kThreads)
        m.node[i] = a.node_info[i];
    for (uint32_t i = tid; i < a.n_top * kStrip * 48; i += kThreads) {
        const uint32_t t = i / (kStrip * 48), rest = i - t * kStrip * 48, loc = rest / 48, cv = rest - loc * 48;
        m.top[t * kSlab + loc * kLS + cv] = loc < nl ? a.top[((size_t)t * a.nloc + b0 + loc) * 48 + cv] : 0;
    }
    for (uint32_t i = tid; i < a.n_int * kSlab / 2; i += kThreads)
        reinterpret_cast<uint32_t *>(m.inter)[i] = 0;
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

    // ---- phase 2: internal nodes, decoded, then reconstructed level by level
    if (a.n_int > 0) {
        const uint32_t cnt = build_list(a, m, 0, a.n_int, &s_count, false);
        decode_list<OffT>(a, m, s_mode, cnt, rs, 0, m.inter);
        __syncthreads();
        for (uint32_t p0 = 0; p0 < a.n_int;) {
            const uint32_t lvl = node_level(m.node[p0]);
            uint32_t p1 = p0;
            while (p1 < a.n_int && node_level(m.node[p1]) == lvl)
                p1++;
            const bool from_top = lvl + 2 == a.L;
            for (uint32_t i = tid; i < (p1 - p0) * kSlab; i += kThreads) {
                const uint32_t p = p0 + i / kSlab, rest = i % kSlab;
                const uint32_t par = node_parent(m.node[p]);
                const int16_t *src = from_top ? m.top : m.inter;
                m.inter[p * kSlab + rest] += src[par * kSlab + rest];
            }
            __syncthreads();
            p0 = p1;
        }
    }

    // ---- phase 3: the views, in batches of up to kLeafMax views whose stored
    // blocks fit the kResCap decode slots
    const bool use_mask = kPacked && a.needed != nullptr;
    for (uint32_t p = a.n_int + tid; p < a.S; p += kThreads) {
        uint32_t cnt = 0;
        if (!use_mask || a.needed[node_view(m.node[p])])
            for (uint32_t r = 0; r < kRecs; r++)
                cnt += (m.mask[r * a.MW + (p >> 5)] >> (p & 31u)) & 1u;
        m.leafcnt[p - a.n_int] = (uint16_t)cnt;
    }
    __shared__ uint32_t s_p1;
    for (uint32_t p0 = a.n_int; p0 < a.S;) {
        __syncthreads();
        if (warp == 0) {
            // the longest run of views from p0 whose stored blocks fit
            uint32_t sum = 0, p1 = p0;
            const uint32_t lim = min(a.S, p0 + kLeafMax);
            for (uint32_t q0 = p0; q0 < lim; q0 += 32) {
                const uint32_t q = q0 + lane;
                const uint32_t c = q < lim ? m.leafcnt[q - a.n_int] : (uint32_t)kResCap + 1;
                const uint32_t incl = warp_inclusive_scan(c, lane);
                const unsigned ok = __ballot_sync(kFullMask, sum + incl <= (uint32_t)kResCap);
                const uint32_t n_ok = __popc(ok);
                if (n_ok)
                    sum += __shfl_sync(kFullMask, incl, n_ok - 1);
                p1 = q0 + n_ok;
                if (n_ok < 32)
                    break;
            }
            if (lane == 0)
                s_p1 = max(p1, p0 + 1);
        }
        __syncthreads();
        const uint32_t p1 = s_p1, nb = p1 - p0;
        const uint32_t cnt = build_leaf_list(a, m, p0, p1, &s_count, use_mask);
        decode_leaf_list<OffT>(a, m, s_mode, cnt, rs);
        __syncthreads();
        // parent + residual -> RGB: one (view, kRowsPerJob block rows) per
        // warp step, lane = (row, location), four pixels per lane written
        // straight to the output row
        constexpr uint32_t kJobsPerView = 4 / kRowsPerJob;
        for (uint32_t job = warp; job < nb * kJobsPerView; job += kWarps) {
            const uint32_t j = job / kJobsPerView;
            const uint32_t info = m.node[p0 + j];
            const uint32_t view = node_view(info);
            if (use_mask && !a.needed[view])
                continue;
            const uint32_t row = (job % kJobsPerView) * kRowsPerJob + lane / kStrip, loc = lane % kStrip;
            const uint32_t y = by * 4 + row, x = (bx0 + loc) * 4;
            if (loc >= nl || y >= a.H)
                continue;
            const int16_t *base = (a.L == 2 ? m.top : m.inter) + node_parent(info) * kSlab + loc * kLS + row * 4;
            int32_t ycc[3][4];
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const uint2 pb = *reinterpret_cast<const uint2 *>(base + c * 16);
                const uint32_t slot = m.map[j * kRecs + loc * 3 + c];
                const uint2 rb = slot != 0xFFFFu ? *reinterpret_cast<const uint2 *>(m.res + slot * kVals + row * 4)
                                                 : make_uint2(0u, 0u);
                ycc[c][0] = (int32_t)(int16_t)(pb.x & 0xFFFFu) + (int32_t)(int16_t)(rb.x & 0xFFFFu);
                ycc[c][1] = (int32_t)(int16_t)(pb.x >> 16) + (int32_t)(int16_t)(rb.x >> 16);
                ycc[c][2] = (int32_t)(int16_t)(pb.y & 0xFFFFu) + (int32_t)(int16_t)(rb.y & 0xFFFFu);
                ycc[c][3] = (int32_t)(int16_t)(pb.y >> 16) + (int32_t)(int16_t)(rb.y >> 16);
            }
            uint32_t px[4];
#pragma unroll
            for (int k = 0; k < 4; k++)
                px[k] = ycocg_to_rgb24(ycc[0][k], ycc[1][k], ycc[2][k]);
            const bool whole = x + 4 <= a.W;
            if (kPacked) {
                uint32_t *dst = reinterpret_cast<uint32_t *>(a.out) + ((size_t)view * a.H + y) * a.W + x;
                if (whole && a.out_aligned16 && (a.W & 3u) == 0) {
                    *reinterpret_cast<uint4 *>(dst) = make_uint4(px[0], px[1], px[2], px[3]);
                } else {
                    for (uint32_t k = 0; k < 4 && x + k < a.W; k++)
                        dst[k] = px[k];
                }
            } else {
                uint8_t *dst = a.out + (((size_t)view * a.H + y) * a.W + x) * 3;
                if (whole && a.out_aligned4 && (a.W & 3u) == 0) {
                    // 4 pixels = 12 bytes = 3 words at a 4-byte boundary, each
                    // assembled by one byte permute of two neighbouring pixels
                    uint32_t *d = reinterpret_cast<uint32_t *>(dst);
                    d[0] = __byte_perm(px[0], px[1], 0x4210);
                    d[1] = __byte_perm(px[1], px[2], 0x5421);
                    d[2] = __byte_perm(px[2], px[3], 0x6542);
                } else {
                    for (uint32_t k = 0; k < 4 && x + k < a.W; k++) {
                        dst[3 * k] = (uint8_t)px[k];
                        dst[3 * k + 1] = (uint8_t)(px[k] >> 8);
                        dst[3 * k + 2] = (uint8_t)(px[k] >> 16);
                    }
                }
            }
        }
        p0 = p1;
    }
}

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
    return launch_decode<false>(s, d_out, nullptr, st);
}

int launch_decode_packed(const rlfc_stream *s, uint32_t *d_out, const uint8_t *needed, cudaStream_t st)
{
    return launch_decode<true>(s, reinterpret_cast<uint8_t *>(d_out), needed, st);
}

}  // namespace rlfc

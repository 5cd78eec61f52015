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
//  3. the views (leaves), kLeafBatch at a time: compacted, decoded the same
//     way into a residual buffer, then parent + residual is converted from
//     YCoCg-R to RGB and written as whole image rows with 16-byte stores.
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

constexpr int kStrip = 16;       // block locations per CTA
constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kLeafBatch = 16;
constexpr int kRecs = 3 * kStrip;
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
    uint32_t pmax;          // largest number of stored blocks in one record
    uint32_t list_cap;      // work-list capacity (items)
};

struct Smem {
    uint32_t *node;    // [S]
    int16_t *top;      // [n_top][48][kStrip]
    int16_t *inter;    // [n_int][48][kStrip]  internal reconstructions
    int16_t *res;      // [kLeafBatch][48][kStrip]  leaf residuals
    uint8_t *rgb;      // [kWarps][row bytes]: one output row per warp
    uint32_t *mask;    // [kRecs][MW]
    void *off;         // [kRecs][pmax]  payload bit offset of each stored block (OffT)
    uint2 *list;       // [list_cap]  (node | record << 16, rank)
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
    p += r16(2ull * a.n_top * 48 * kStrip);
    m.inter = reinterpret_cast<int16_t *>(p);
    p += r16(2ull * a.n_int * 48 * kStrip);
    m.res = reinterpret_cast<int16_t *>(p);
    p += r16(2ull * kLeafBatch * 48 * kStrip);
    m.rgb = p;
    p += r16((size_t)kWarps * kStrip * 16);
    m.mask = reinterpret_cast<uint32_t *>(p);
    p += r16(4ull * kRecs * a.MW);
    m.off = p;
    p += r16(sizeof(OffT) * kRecs * a.pmax);
    m.list = reinterpret_cast<uint2 *>(p);
    return m;
}

inline size_t smem_bytes(uint32_t S, uint32_t n_top, uint32_t n_int, uint32_t MW, uint32_t pmax, uint32_t list_cap,
                         size_t off_size)
{
    return r16(4ull * S) + r16(2ull * n_top * 48 * kStrip) + r16(2ull * n_int * 48 * kStrip) +
           r16(2ull * kLeafBatch * 48 * kStrip) + r16((size_t)kWarps * kStrip * 16) +
           r16(4ull * kRecs * MW) + r16(off_size * kRecs * pmax) + r16(8ull * list_cap);
}

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
            const uint32_t *mk = m.mask + r * a.MW;
            present = (mk[p >> 5] >> (p & 31u)) & 1u;
            if (present && use_mask)
                present = a.needed[node_view(m.node[p])] != 0;
            if (present) {
                for (uint32_t w = 0; w < (p >> 5); w++)
                    rank += __popc(mk[w]);
                rank += __popc(mk[p >> 5] & ((1u << (p & 31u)) - 1u));
            }
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

// Decode the listed blocks, one block per thread; the residual
// (min + u) * 2^(q + shift) goes to the node's slot in dst:
// dst[((node - p0) * 48 + channel * 16 + value) * kStrip + location].
template <typename OffT>
__device__ __forceinline__ void decode_list(const Args &a, const Smem &m, const uint32_t *s_mode, uint32_t count,
                                            uint32_t b0, uint32_t p0, int16_t *dst)
{
    const OffT *off = reinterpret_cast<const OffT *>(m.off);
    const uint32_t hdr0 = 32 * a.MW;
    for (uint32_t i = threadIdx.x; i < count; i += kThreads) {
        const uint2 it = m.list[i];
        const uint32_t p = it.x & 0xFFFFu, r = it.x >> 16, rank = it.y;
        const uint32_t loc = r / 3, c = r - 3 * loc;
        const uint32_t *rec = a.records + a.offsets[3 * b0 + r];
        const BlockHeader h = unpack_header(get_bits(rec, hdr0 + kHdrBits * rank, kHdrBits));
        int32_t u[kVals];
        bise_decode16(rec, off[r * a.pmax + rank], s_mode[h.mode], u);
        const int32_t scale = 1 << (a.q + h.shift);
        int16_t *d = dst + ((p - p0) * 48 + c * 16) * kStrip + loc;
#pragma unroll
        for (int v = 0; v < kVals; v++)
            d[v * kStrip] = (int16_t)((h.min + u[v]) * scale);
    }
}

template <bool kPacked, typename OffT>
__global__ void __launch_bounds__(kThreads) decode_all_kernel(const Args a)
{
    constexpr uint32_t kRowBytes = kPacked ? kStrip * 16 : kStrip * 12;
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
        m.top[(t * 48 + cv) * kStrip + loc] = loc < nl ? a.top[((size_t)t * a.nloc + b0 + loc) * 48 + cv] : 0;
    }
    for (uint32_t i = tid; i < a.n_int * 48 * kStrip / 2; i += kThreads)
        reinterpret_cast<uint32_t *>(m.inter)[i] = 0;
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
        const uint32_t *rec = a.records + a.offsets[3 * b0 + r];
        uint32_t P = 0;
        for (uint32_t w0 = 0; w0 < a.MW; w0 += 32) {
            const uint32_t word = w0 + lane < a.MW ? rec[w0 + lane] : 0u;
            if (w0 + lane < a.MW)
                mk[w0 + lane] = word;
            P += __reduce_add_sync(kFullMask, (uint32_t)__popc(word));
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
        decode_list<OffT>(a, m, s_mode, cnt, b0, 0, m.inter);
        __syncthreads();
        for (uint32_t p0 = 0; p0 < a.n_int;) {
            const uint32_t lvl = node_level(m.node[p0]);
            uint32_t p1 = p0;
            while (p1 < a.n_int && node_level(m.node[p1]) == lvl)
                p1++;
            const bool from_top = lvl + 2 == a.L;
            for (uint32_t i = tid; i < (p1 - p0) * 48 * kStrip; i += kThreads) {
                const uint32_t p = p0 + i / (48 * kStrip), rest = i % (48 * kStrip);
                const uint32_t par = node_parent(m.node[p]);
                const int16_t *src = from_top ? m.top : m.inter;
                m.inter[p * 48 * kStrip + rest] += src[par * 48 * kStrip + rest];
            }
            __syncthreads();
            p0 = p1;
        }
    }

    // ---- phase 3: the views, kLeafBatch at a time
    const bool fast_rows = a.out_aligned16 && (a.W % (kPacked ? 4 : 16) == 0) && nl == kStrip &&
                           bx0 * 4 + kStrip * 4 <= a.W;
    for (uint32_t p0 = a.n_int; p0 < a.S; p0 += kLeafBatch) {
        const uint32_t nb = min((uint32_t)kLeafBatch, a.S - p0);
        for (uint32_t i = tid; i < kLeafBatch * 48 * kStrip / 2; i += kThreads)
            reinterpret_cast<uint32_t *>(m.res)[i] = 0;
        const uint32_t cnt = build_list(a, m, p0, p0 + nb, &s_count, kPacked && a.needed != nullptr);
        decode_list<OffT>(a, m, s_mode, cnt, b0, p0, m.res);
        __syncthreads();
        // parent + residual -> RGB, one (leaf, pixel row) per warp step;
        // lane = (location, pixel pair)
        for (uint32_t job = warp; job < nb * 4; job += kWarps) {
            const uint32_t j = job >> 2, row = job & 3;
            const uint32_t info = m.node[p0 + j];
            const uint32_t view = node_view(info);
            if (kPacked && a.needed && !a.needed[view])
                continue;
            const uint32_t par = node_parent(info);
            const int16_t *base = (a.L == 2 ? m.top : m.inter) + par * 48 * kStrip;
            const int16_t *rs = m.res + j * 48 * kStrip;
            uint8_t *srow = m.rgb + warp * kRowBytes;
            const uint32_t loc = lane >> 1, x2 = (lane & 1) * 2;
            if (loc < nl) {
                uint32_t px[2];
#pragma unroll
                for (int x = 0; x < 2; x++) {
                    const uint32_t k = row * 4 + x2 + x;
                    const int yy = base[k * kStrip + loc] + rs[k * kStrip + loc];
                    const int co = base[(16 + k) * kStrip + loc] + rs[(16 + k) * kStrip + loc];
                    const int cg = base[(32 + k) * kStrip + loc] + rs[(32 + k) * kStrip + loc];
                    px[x] = ycocg_to_rgb24(yy, co, cg);
                }
                if (kPacked) {
                    reinterpret_cast<uint2 *>(srow)[lane] = make_uint2(px[0], px[1]);
                } else {
                    uint16_t *w = reinterpret_cast<uint16_t *>(srow + lane * 6);
                    w[0] = (uint16_t)px[0];
                    w[1] = (uint16_t)((px[0] >> 16) | (px[1] << 8));
                    w[2] = (uint16_t)(px[1] >> 8);
                }
            }
            __syncwarp();
            const uint32_t y = by * 4 + row, x0 = bx0 * 4;
            if (y < a.H && x0 < a.W) {
                if (kPacked) {
                    uint32_t *dst = reinterpret_cast<uint32_t *>(a.out) + ((size_t)view * a.H + y) * a.W + x0;
                    const uint32_t *src = reinterpret_cast<const uint32_t *>(srow);
                    if (fast_rows) {
                        if (lane < kStrip)
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
    a.pmax = std::max<uint32_t>(s->max_present, 1);
    a.list_cap = kRecs * std::max<uint32_t>(t.n_int, kLeafBatch);
    // payload offsets are bit positions inside one record: 16 bits suffice
    // unless a record reaches 2^16 bits
    const bool off16 = (uint64_t)s->max_record_words * 32 < 65536;
    const size_t smem = smem_bytes(a.S, a.n_top, a.n_int, a.MW, a.pmax, a.list_cap, off16 ? 2 : 4);
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

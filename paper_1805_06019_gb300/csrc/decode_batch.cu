// Batched random-access block decode: Algorithm 2's DecompressLFIBlock for
// many (view, location) requests in one call, with the progressive stop level
// of Section 3.6.
//
// The requests are grouped by block location with a counting sort (count,
// scan, scatter), then a persistent kernel serves the locations.  Its warps
// take locations from an atomic work queue (no waits: a warp that finds the
// queue empty exits).  For each location a warp
//   1. optionally copies the location's three channel records (they are
//      contiguous in the stream) into its shared-memory slice, or has them
//      copied there ahead of time (cp.async) while it serves the previous
//      location;
//   2. parses each record once: presence-mask popcount prefixes, then the
//      closed-form payload length of every stored block from its 5-bit mode,
//      turned into payload bit offsets by a warp scan;
//   3. for up to kSlots requests at a time: seeds int32 accumulators with the
//      top-RKV block, lists the stored ancestor blocks (request, channel,
//      level) with a ballot compaction, decodes them one thread per block
//      with the sequential bit reader and adds (min + u) 2^(q + s) into the
//      accumulators, converts YCoCg-R to clamped RGB and writes 48 bytes per
//      request.
// The record gather (mask, headers, offsets) is paid once per location and
// shared by every request there, which is the point of batching.
#include <cuda_runtime.h>

#include <cuda_pipeline.h>

#include <algorithm>
#include <new>

#include "rlfc_device.cuh"
#include "rlfc_internal.h"

namespace rlfc {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr uint32_t kSlots = 8;          // requests of one location per round
constexpr uint32_t kStageCap = 1024;    // words of records staged per warp at most
constexpr uint32_t kBadRank = 0xFFFFFFFFu;

__constant__ uint32_t c_modes[kNumModes] = RLFC_MODE_TABLE_INIT;

__device__ __forceinline__ uint32_t scan_incl(uint32_t x, int lane)
{
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, x, d);
        if (lane >= d)
            x += y;
    }
    return x;
}

struct BinArgs {
    const uint32_t *view;
    const uint32_t *loc;
    uint8_t *out;
    uint8_t *status;
    uint32_t *cnt;      // [nloc + 2]: counts, then bin starts; [nloc + 1] is the queue head,
                        // followed by the scan's per-chunk counts
    uint32_t *rank;     // [n]: position of the request inside its bin
    uint32_t *sorted;   // [n]: request indices grouped by location
    uint32_t *sorted_view;  // [n]: their views, in the same order
    uint32_t n, n_views, nloc, aligned;
};

// Validate, count per location, remember the position inside the bin.
__global__ void bin_count_kernel(const BinArgs a)
{
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= a.n)
        return;
    const uint32_t view = a.view[r], loc = a.loc[r];
    const uint32_t bad = view >= a.n_views ? (uint32_t)RLFC_REQ_BAD_VIEW
                                           : (loc >= a.nloc ? (uint32_t)RLFC_REQ_BAD_LOCATION : 0u);
    if (a.status)
        a.status[r] = (uint8_t)bad;
    if (bad) {
        uint8_t *dst = a.out + (size_t)r * 48;
        if (a.aligned) {
            for (int w = 0; w < 12; w++)
                reinterpret_cast<uint32_t *>(dst)[w] = 0u;
        } else {
            for (int b = 0; b < 48; b++)
                dst[b] = 0;
        }
        a.rank[r] = kBadRank;
        return;
    }
    a.rank[r] = atomicAdd(&a.cnt[loc], 1u);
}

constexpr uint32_t kScanChunk = 4096;   // locations per CTA of the scan (1024 threads x 4)

__device__ __forceinline__ uint32_t block_sum(uint32_t x, uint32_t *s_warp)
{
    const int lane = (int)(threadIdx.x & 31u);
    x = __reduce_add_sync(kFull, x);
    if (lane == 0)
        s_warp[threadIdx.x >> 5] = x;
    __syncthreads();
    const uint32_t r = __reduce_add_sync(kFull, lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0u);
    __syncthreads();
    return r;
}

// Scan, pass 1: the request count of every chunk of kScanChunk locations.
__global__ void __launch_bounds__(1024) bin_reduce_kernel(const uint32_t *cnt, uint32_t nloc, uint32_t *part)
{
    __shared__ uint32_t s_warp[32];
    const uint32_t base = blockIdx.x * kScanChunk;
    uint32_t x = 0;
#pragma unroll
    for (uint32_t k = 0; k < 4; k++) {
        const uint32_t i = base + k * 1024 + threadIdx.x;
        x += i < nloc ? cnt[i] : 0u;
    }
    x = block_sum(x, s_warp);
    if (threadIdx.x == 0)
        part[blockIdx.x] = x;
}

// Scan, pass 2: exclusive scan of cnt[0..nloc) in place, chunk by chunk in
// parallel (each chunk starts at the sum of the chunks before it);
// cnt[nloc] = total.
__global__ void __launch_bounds__(1024) bin_scan_kernel(uint32_t *cnt, uint32_t nloc, const uint32_t *part)
{
    __shared__ uint32_t s_warp[32];
    const int lane = (int)(threadIdx.x & 31u);
    const uint32_t warp = threadIdx.x >> 5;
    uint32_t before = 0;
    for (uint32_t c = threadIdx.x; c < blockIdx.x; c += 1024)
        before += part[c];
    before = block_sum(before, s_warp);
    // four consecutive locations per thread
    const uint32_t i0 = blockIdx.x * kScanChunk + 4 * threadIdx.x;
    uint32_t v[4];
#pragma unroll
    for (uint32_t k = 0; k < 4; k++)
        v[k] = i0 + k < nloc ? cnt[i0 + k] : 0u;
    const uint32_t sum = v[0] + v[1] + v[2] + v[3];
    const uint32_t incl = scan_incl(sum, lane);
    if (lane == 31)
        s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const uint32_t x = s_warp[lane];
        s_warp[lane] = scan_incl(x, lane) - x;
    }
    __syncthreads();
    uint32_t run = before + s_warp[warp] + incl - sum;
#pragma unroll
    for (uint32_t k = 0; k < 4; k++) {
        if (i0 + k < nloc)
            cnt[i0 + k] = run;
        run += v[k];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 1023)
        cnt[nloc] = run;
}

__global__ void bin_scatter_kernel(const BinArgs a)
{
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= a.n)
        return;
    const uint32_t rk = a.rank[r];
    if (rk != kBadRank) {
        const uint32_t at = a.cnt[a.loc[r]] + rk;
        a.sorted[at] = r;
        a.sorted_view[at] = a.view[r];
    }
}

struct DecArgs {
    const uint32_t *records;
    const uint32_t *offsets;
    const int16_t *top;       // [n_top][nloc][48]
    const uint32_t *view_anc; // [n_views][kMaxLevels]
    const uint32_t *req_view;
    const uint32_t *start;    // [nloc + 1] bin starts
    const uint32_t *sorted;
    const uint32_t *sorted_view;
    uint8_t *out;
    uint32_t *queue;
    uint32_t nloc, L, q, MW, level, pmax, locs_per_pop, stage, stage_words, warp_words, aligned;
    uint32_t anc_words;       // view_anc words cached in shared memory (0: read it from global)
    uint32_t *dbg;            // debug builds: the stream's flag word
};

// Per-warp shared-memory words for a configuration (the CTA adds the cached
// ancestor table after its warps' slices).
// stage: 0 none, 1 one buffer, 2 two buffers (prefetch); each buffer holds
// stage_words + 4 words.
__host__ __device__ inline uint32_t warp_words_for(uint32_t MW, uint32_t pmax, uint32_t L, uint32_t stage,
                                                   uint32_t stage_words)
{
    const uint32_t w = 6 * MW + 3 * pmax + kSlots * 48 + 2 * kSlots + kSlots * 3 * (L - 1) + kSlots * 16 +
                       stage * (stage_words + 4);
    return (w + 3u) & ~3u;
}

__global__ void __launch_bounds__(512) decode_binned_kernel(const DecArgs a)
{
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ uint32_t s_modes[kNumModes];
    if (threadIdx.x < kNumModes)
        s_modes[threadIdx.x] = c_modes[threadIdx.x];
    // the ancestor table, shared by the CTA's warps when it is small
    const uint32_t *view_anc = a.view_anc;
    if (a.anc_words) {
        uint32_t *s_anc = smem + (blockDim.x >> 5) * a.warp_words;
        for (uint32_t i = threadIdx.x; i < a.anc_words; i += blockDim.x)
            s_anc[i] = a.view_anc[i];
        view_anc = s_anc;
    }
    __syncthreads();
    const int lane = (int)(threadIdx.x & 31u);
    uint32_t *s_mask = smem + (threadIdx.x >> 5) * a.warp_words;   // [3][MW]
    uint32_t *s_mpre = s_mask + 3 * a.MW;                           // [3][MW] popcount before each word
    uint32_t *s_off = s_mpre + 3 * a.MW;                            // [3][pmax] payload bit offsets
    int32_t *s_acc = reinterpret_cast<int32_t *>(s_off + 3 * a.pmax);   // [kSlots][3][16]
    uint32_t *s_req = reinterpret_cast<uint32_t *>(s_acc + kSlots * 48);
    uint32_t *s_view = s_req + kSlots;
    uint32_t *s_list = s_view + kSlots;                             // [kSlots * 3 * (L-1)]
    uint32_t *s_rgb = s_list + kSlots * 3 * (a.L - 1);              // [kSlots][16]
    uint32_t *s_stage = s_rgb + kSlots * 16;
    const uint32_t nl = a.L - 1 - a.level;   // SRV levels added to the top RKV
    const uint32_t hdr0 = 32 * a.MW;

    // One location: parse its three records (from `staged` when they were
    // copied to shared memory, else from the stream) and serve its requests.
    auto serve = [&](uint32_t loc, const uint32_t *staged) {
        {
            const uint32_t r0 = a.start[loc], r1 = a.start[loc + 1];
            if (r0 == r1)
                return;
            const uint32_t o0 = a.offsets[3 * loc];
            const uint32_t d1 = a.offsets[3 * loc + 1] - o0, d2 = a.offsets[3 * loc + 2] - o0;
            const uint32_t span = a.offsets[3 * loc + 3] - o0;
            const uint32_t *base = staged ? staged : a.records + o0;
            if (!staged && a.stage == 1 && span <= a.stage_words) {
                // the bit reader may touch one word past a record: copy two more
                // (the stream carries zero padding after its last record)
                for (uint32_t i = lane; i < span + 2; i += 32)
                    s_stage[i] = base[i];
                __syncwarp();
                base = s_stage;
            }
            // parse the three records
#pragma unroll
            for (uint32_t c = 0; c < 3; c++) {
                const uint32_t *rc = base + (c == 0 ? 0u : (c == 1 ? d1 : d2));
                uint32_t total = 0;
                for (uint32_t w0 = 0; w0 < a.MW; w0 += 32) {
                    const uint32_t wi = w0 + lane;
                    const uint32_t word = wi < a.MW ? rc[wi] : 0u;
                    const uint32_t cnt = __popc(word);
                    const uint32_t incl = scan_incl(cnt, lane);
                    if (wi < a.MW) {
                        s_mask[c * a.MW + wi] = word;
                        s_mpre[c * a.MW + wi] = total + incl - cnt;
                    }
                    total += __shfl_sync(kFull, incl, 31);
                }
                const uint32_t pay0 = hdr0 + kHdrBits * total;
                uint32_t run = 0;
                for (uint32_t h0 = 0; h0 < total; h0 += 32) {
                    const uint32_t hi = h0 + lane;
                    const uint32_t len = hi < total ? mode_bits(s_modes[get_bits(rc, hdr0 + kHdrBits * hi, 5)]) : 0u;
                    const uint32_t incl = scan_incl(len, lane);
                    if (hi < total)
                        s_off[c * a.pmax + hi] = pay0 + run + incl - len;
                    run += __shfl_sync(kFull, incl, 31);
                }
            }
            __syncwarp();
            for (uint32_t j0 = r0; j0 < r1; j0 += kSlots) {
                const uint32_t ns = min(kSlots, r1 - j0);
                if ((uint32_t)lane < ns) {
                    s_req[lane] = a.sorted[j0 + lane];
                    s_view[lane] = a.sorted_view[j0 + lane];
                }
                __syncwarp();
                // ReadBlock(RKV^n, BlkIdx): the accumulators start at the top RKV
                // (96 bytes per slot, as six 16-byte loads)
                for (uint32_t i = lane; i < ns * 6; i += 32) {
                    const uint32_t slot = i / 6, k = i - slot * 6;
                    const uint32_t top = view_anc[s_view[slot] * kMaxLevels + a.L - 1];
                    const uint4 v = reinterpret_cast<const uint4 *>(a.top + ((size_t)top * a.nloc + loc) * 48)[k];
                    int32_t *d = s_acc + slot * 48 + k * 8;
                    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        d[2 * e] = (int32_t)(int16_t)(w[e] & 0xFFFFu);
                        d[2 * e + 1] = (int32_t)w[e] >> 16;
                    }
                }
                // stored ancestor blocks of these requests, compacted
                const uint32_t ntask = ns * 3 * nl;
                uint32_t cnt = 0;
                for (uint32_t t0 = 0; t0 < ntask; t0 += 32) {
                    const uint32_t t = t0 + lane;
                    uint32_t code = 0;
                    bool pres = false;
                    if (t < ntask) {
                        const uint32_t slot = t / (3 * nl), rem = t - slot * 3 * nl;
                        const uint32_t c = rem / nl, l = a.level + (rem - c * nl);
                        const uint32_t node = view_anc[s_view[slot] * kMaxLevels + l];
                        const uint32_t wi = node >> 5, bit = node & 31u;
                        const uint32_t word = s_mask[c * a.MW + wi];
                        pres = (word >> bit) & 1u;
                        const uint32_t rank = s_mpre[c * a.MW + wi] + __popc(word & ((1u << bit) - 1u));
                        code = rank | (c << 16) | (slot << 18);
                    }
                    const uint32_t bal = __ballot_sync(kFull, pres);
                    if (pres)
                        s_list[cnt + __popc(bal & ((1u << lane) - 1u))] = code;
                    cnt += __popc(bal);
                }
                __syncwarp();
                // BISEDecode + CombineBlocks, one thread per stored block
                for (uint32_t i = lane; i < cnt; i += 32) {
                    const uint32_t code = s_list[i];
                    const uint32_t rank = code & 0xFFFFu, c = (code >> 16) & 3u, slot = code >> 18;
                    const uint32_t *rc = base + (c == 0 ? 0u : (c == 1 ? d1 : d2));
                    const BlockHeader h = unpack_header(get_bits(rc, hdr0 + kHdrBits * rank, kHdrBits));
#ifdef RLFC_DEBUG
                    {
                        const uint32_t rec_words = c == 0 ? d1 : (c == 1 ? d2 - d1 : span - d2);
                        const uint32_t P = s_mpre[c * a.MW + a.MW - 1] + __popc(s_mask[c * a.MW + a.MW - 1]);
                        if (!RLFC_DBG_BLOCK_OK(a.dbg, h.mode, hdr0 + kHdrBits * (rank + 1), hdr0 + kHdrBits * P,
                                               s_off[c * a.pmax + rank],
                                               h.mode < (uint32_t)kNumModes ? mode_bits(s_modes[h.mode]) : 0u,
                                               32u * rec_words))
                            continue;
                    }
#endif
                    int32_t u[kVals];
                    bise_decode16(rc, s_off[c * a.pmax + rank], s_modes[h.mode], u);
                    const int32_t scale = 1 << (a.q + h.shift);
                    int32_t *dst = s_acc + slot * 48 + c * 16;
#pragma unroll
                    for (int v = 0; v < kVals; v++)
                        atomicAdd(&dst[v], (h.min + u[v]) * scale);
                }
                __syncwarp();
                for (uint32_t i = lane; i < ns * 16; i += 32) {
                    const uint32_t slot = i >> 4, k = i & 15u;
                    const int32_t *acc = s_acc + slot * 48;
                    s_rgb[i] = ycocg_to_rgb24(acc[k], acc[16 + k], acc[32 + k]);
                }
                __syncwarp();
                if (a.aligned) {
                    // 48 bytes as 12 words; word w starts at byte (4w) % 3 of
                    // pixel (4w) / 3 and ends inside the next pixel
                    for (uint32_t i = lane; i < ns * 12; i += 32) {
                        const uint32_t slot = i / 12, wd = i - slot * 12;
                        const uint32_t p0 = (4 * wd) / 3;
                        const uint32_t lo = s_rgb[slot * 16 + p0], hi = s_rgb[slot * 16 + p0 + 1];
                        const uint32_t sh = (4 * wd) % 3;   // first byte of the word inside pixel p0
                        reinterpret_cast<uint32_t *>(a.out + (size_t)s_req[slot] * 48)[wd] =
                            __byte_perm(lo, hi, sh == 0 ? 0x4210u : (sh == 1 ? 0x5421u : 0x6542u));
                    }
                } else {
                    for (uint32_t i = lane; i < ns * 48; i += 32) {
                        const uint32_t slot = i / 48, byte = i - slot * 48;
                        a.out[(size_t)s_req[slot] * 48 + byte] = (uint8_t)(s_rgb[slot * 16 + byte / 3] >> (8 * (byte % 3)));
                    }
                }
                __syncwarp();
            }
        }
    };

    if (a.stage == 2) {
        // prefetching: while a location is served, the records of the next
        // one are copied into the warp's other buffer (cp.async)
        uint32_t *const buf0 = s_stage, *const buf1 = s_stage + a.stage_words + 4;
        auto pop = [&]() {
            uint32_t v = 0;
            if (lane == 0)
                v = atomicAdd(a.queue, 1u);
            return __shfl_sync(kFull, v, 0);
        };
        auto prefetch = [&](uint32_t loc, uint32_t *dst) {
            if (loc >= a.nloc)
                return false;
            const uint32_t o0 = a.offsets[3 * loc], span = a.offsets[3 * loc + 3] - o0;
            if (span > a.stage_words)
                return false;
            for (uint32_t i = lane; i < span + 2; i += 32)
                __pipeline_memcpy_async(dst + i, a.records + o0 + i, 4);
            return true;
        };
        uint32_t cur = pop();
        bool cur_in = prefetch(cur, buf0);
        __pipeline_commit();
        uint32_t parity = 0;
        while (cur < a.nloc) {
            const uint32_t nxt = pop();
            const bool nxt_in = prefetch(nxt, parity ? buf0 : buf1);
            __pipeline_commit();
            __pipeline_wait_prior(1);   // this lane's copies of `cur` are done
            __syncwarp();               // and every lane's
            serve(cur, cur_in ? (parity ? buf1 : buf0) : nullptr);
            __syncwarp();               // the buffer is free for the prefetch after next
            cur = nxt;
            cur_in = nxt_in;
            parity ^= 1u;
        }
        __pipeline_wait_prior(0);
        return;
    }
    for (;;) {
        uint32_t first = 0;
        if (lane == 0)
            first = atomicAdd(a.queue, a.locs_per_pop);
        first = __shfl_sync(kFull, first, 0);
        if (first >= a.nloc)
            break;
        const uint32_t last = min(first + a.locs_per_pop, a.nloc);
        for (uint32_t loc = first; loc < last; loc++)
            serve(loc, nullptr);
    }
}

bool valid_config(const rlfc_batch_config &c)
{
    return (c.warps_per_cta == 4 || c.warps_per_cta == 8 || c.warps_per_cta == 16) && c.locs_per_pop >= 1 &&
           c.locs_per_pop <= 64 && c.stage <= 2 && c.graph <= 1;
}

}  // namespace
}  // namespace rlfc

struct rlfc_batch {
    const rlfc_stream *s = nullptr;
    int device = 0;
    size_t max_n = 0;
    uint32_t nloc = 0, pmax = 1, stage_words = 0, smem_optin = 0, sms = 0;
    uint32_t *d_cnt = nullptr;      // nloc + 2 words, then one per scan chunk
    uint32_t *d_rank = nullptr;     // max_n
    uint32_t *d_sorted = nullptr;   // max_n
    uint32_t *d_sorted_view = nullptr;   // max_n
    uint32_t anc_words = 0;         // ancestor-table words cached per CTA (0 = none)
    rlfc_batch_config cfg{8, 1, 0, 1};
    cudaStream_t cap = nullptr;     // private stream, only ever capturing
    cudaGraphExec_t exec = nullptr;
    struct Key {
        const void *view, *loc, *out, *status;
        size_t n;
        uint32_t level;
        bool operator==(const Key &o) const
        {
            return view == o.view && loc == o.loc && out == o.out && status == o.status && n == o.n &&
                   level == o.level;
        }
    } key{};
};

namespace rlfc {
namespace {

uint32_t smem_bytes(const rlfc_batch *b, const rlfc_batch_config &c)
{
    return c.warps_per_cta * 4u * warp_words_for(b->s->MW, b->pmax, b->s->tab.L, c.stage, b->stage_words) +
           4u * b->anc_words;
}

bool fits(const rlfc_batch *b, const rlfc_batch_config &c) { return smem_bytes(b, c) <= b->smem_optin; }

int enqueue(rlfc_batch *b, const rlfc_batch_config &cfg, const uint32_t *view, const uint32_t *loc, uint32_t n,
            uint32_t level, uint8_t *out, uint8_t *status, cudaStream_t st)
{
    const rlfc_stream *s = b->s;
    cudaError_t e = cudaMemsetAsync(b->d_cnt, 0, (size_t)(b->nloc + 2) * 4, st);
    if (e != cudaSuccess)
        return cuda_fail(e, "batch scratch clear");
    BinArgs ba;
    ba.view = view;
    ba.loc = loc;
    ba.out = out;
    ba.status = status;
    ba.cnt = b->d_cnt;
    ba.rank = b->d_rank;
    ba.sorted = b->d_sorted;
    ba.sorted_view = b->d_sorted_view;
    ba.n = n;
    ba.n_views = s->tab.n_views;
    ba.nloc = b->nloc;
    ba.aligned = ((uintptr_t)out & 3u) == 0;
    const uint32_t g = (n + 255) / 256;
    { TraceScope trace_("bin_count_kernel", st); bin_count_kernel<<<g, 256, 0, st>>>(ba); }
    const uint32_t chunks = (b->nloc + kScanChunk - 1) / kScanChunk;
    uint32_t *part = b->d_cnt + b->nloc + 2;
    { TraceScope trace_("bin_reduce_kernel", st); bin_reduce_kernel<<<chunks, 1024, 0, st>>>(b->d_cnt, b->nloc, part); }
    { TraceScope trace_("bin_scan_kernel", st); bin_scan_kernel<<<chunks, 1024, 0, st>>>(b->d_cnt, b->nloc, part); }
    { TraceScope trace_("bin_scatter_kernel", st); bin_scatter_kernel<<<g, 256, 0, st>>>(ba); }

    DecArgs da;
    da.dbg = s->d_debug;
    da.records = s->d_records;
    da.offsets = s->d_offsets;
    da.top = s->d_top;
    da.view_anc = s->d_view_anc;
    da.req_view = view;
    da.start = b->d_cnt;
    da.sorted = b->d_sorted;
    da.sorted_view = b->d_sorted_view;
    da.anc_words = b->anc_words;
    da.out = out;
    da.queue = b->d_cnt + b->nloc + 1;
    da.nloc = b->nloc;
    da.L = s->tab.L;
    da.q = s->info.q;
    da.MW = s->MW;
    da.level = level;
    da.pmax = b->pmax;
    da.locs_per_pop = cfg.locs_per_pop;
    da.stage = cfg.stage;
    da.stage_words = b->stage_words;
    da.warp_words = warp_words_for(s->MW, b->pmax, s->tab.L, cfg.stage, b->stage_words);
    da.aligned = ba.aligned;
    const uint32_t threads = cfg.warps_per_cta * 32, smem = smem_bytes(b, cfg);
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, decode_binned_kernel, (int)threads, smem);
    if (e != cudaSuccess)
        return cuda_fail(e, "batch occupancy");
    const uint32_t grid = b->sms * (uint32_t)std::max(per_sm, 1);
    { TraceScope trace_("decode_binned_kernel", st); decode_binned_kernel<<<grid, threads, smem, st>>>(da); }
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_fail(e, "batch decode launch");
    return RLFC_OK;
}

void drop_graph(rlfc_batch *b)
{
    if (b->exec)
        cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
}

int check_args(const rlfc_batch *b, const uint32_t *view, const uint32_t *loc, size_t n, uint32_t level,
               const uint8_t *out)
{
    if (!b || (n && (!view || !loc || !out))) {
        set_error("rlfc_batch: null argument");
        return RLFC_E_INVALID_ARG;
    }
    if (level > b->s->tab.L - 1) {
        set_error("rlfc_batch_decode: level must be at most L-1");
        return RLFC_E_INVALID_ARG;
    }
    if (n > b->max_n) {
        set_error("rlfc_batch_decode: more requests than the batch object was created for");
        return RLFC_E_RANGE;
    }
    return RLFC_OK;
}

}  // namespace
}  // namespace rlfc

extern "C" {

RLFC_API int rlfc_batch_create(const rlfc_stream *s, size_t max_requests, rlfc_batch **out)
{
    using namespace rlfc;
    if (!s || !out) {
        set_error("rlfc_batch_create: null argument");
        return RLFC_E_INVALID_ARG;
    }
    *out = nullptr;
    if (max_requests >= (1ull << 31)) {
        set_error("rlfc_batch_create: max_requests must be below 2^31");
        return RLFC_E_RANGE;
    }
    DeviceGuard g(s->device);
    rlfc_batch *b = new (std::nothrow) rlfc_batch;
    if (!b) {
        set_error("rlfc_batch_create: out of host memory");
        return RLFC_E_OOM;
    }
    b->s = s;
    b->device = s->device;
    b->max_n = std::max<size_t>(max_requests, 1);
    b->nloc = s->info.nloc_x * s->info.nloc_y;
    b->pmax = std::max<uint32_t>(s->max_present, 1u);
    b->stage_words = std::min<uint32_t>(3u * s->max_record_words, kStageCap);
    // the ancestor table is cached per CTA up to 1024 views
    b->anc_words = s->tab.n_views <= 1024u ? s->tab.n_views * (uint32_t)kMaxLevels : 0u;
    int v = 0;
    cudaError_t e = cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, s->device);
    b->smem_optin = e == cudaSuccess ? (uint32_t)v : 48u * 1024u;
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, s->device);
    b->sms = (uint32_t)v;
    cudaFuncAttributes fa{};
    if (e == cudaSuccess)
        e = cudaFuncGetAttributes(&fa, decode_binned_kernel);
    if (e == cudaSuccess) {
        // the opt-in limit covers static and dynamic shared memory together
        b->smem_optin -= std::min<uint32_t>(b->smem_optin, (uint32_t)fa.sharedSizeBytes);
        e = cudaFuncSetAttribute(decode_binned_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)b->smem_optin);
    }
    if (e != cudaSuccess) {
        delete b;
        return cuda_fail(e, "rlfc_batch_create");
    }
    rlfc_batch_config c{4, 1, 0, 1};
    if (!fits(b, c)) {
        set_error("rlfc_batch_create: the records' parse state does not fit in shared memory");
        delete b;
        return RLFC_E_UNSUPPORTED;
    }
    if (!fits(b, b->cfg))
        b->cfg = c;
    const size_t chunks = (b->nloc + kScanChunk - 1) / kScanChunk;
    if ((e = cudaMalloc(&b->d_cnt, (size_t)(b->nloc + 2 + chunks) * 4)) != cudaSuccess ||
        (e = cudaMalloc(&b->d_rank, b->max_n * 4)) != cudaSuccess ||
        (e = cudaMalloc(&b->d_sorted, b->max_n * 4)) != cudaSuccess ||
        (e = cudaMalloc(&b->d_sorted_view, b->max_n * 4)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking)) != cudaSuccess) {
        const int rc = e == cudaErrorMemoryAllocation ? RLFC_E_OOM : RLFC_E_CUDA;
        cuda_fail(e, "rlfc_batch_create");
        cudaGetLastError();
        rlfc_batch_free(b);
        return rc;
    }
    *out = b;
    return RLFC_OK;
}

RLFC_API int rlfc_batch_set_config(rlfc_batch *b, const rlfc_batch_config *cfg)
{
    using namespace rlfc;
    if (!b || !cfg || !valid_config(*cfg)) {
        set_error("rlfc_batch_set_config: invalid configuration");
        return RLFC_E_INVALID_ARG;
    }
    if (!fits(b, *cfg)) {
        set_error("rlfc_batch_set_config: configuration needs more shared memory than a CTA has");
        return RLFC_E_UNSUPPORTED;
    }
    DeviceGuard g(b->device);
    drop_graph(b);
    b->cfg = *cfg;
    return RLFC_OK;
}

RLFC_API int rlfc_batch_get_config(const rlfc_batch *b, rlfc_batch_config *cfg)
{
    if (!b || !cfg) {
        rlfc::set_error("rlfc_batch_get_config: null argument");
        return RLFC_E_INVALID_ARG;
    }
    *cfg = b->cfg;
    return RLFC_OK;
}

RLFC_API int rlfc_batch_decode(rlfc_batch *b, const uint32_t *d_view, const uint32_t *d_loc, size_t n,
                               uint32_t level, uint8_t *d_out, uint8_t *d_status, void *cuda_stream)
{
    using namespace rlfc;
    int rc = check_args(b, d_view, d_loc, n, level, d_out);
    if (rc != RLFC_OK || n == 0)
        return rc;
    DeviceGuard g(b->device);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (!b->cfg.graph)
        return enqueue(b, b->cfg, d_view, d_loc, (uint32_t)n, level, d_out, d_status, st);
    const rlfc_batch::Key k{d_view, d_loc, d_out, d_status, n, level};
    if (!b->exec || !(k == b->key)) {
        drop_graph(b);
        cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess)
            return cuda_fail(e, "batch graph capture");
        rc = enqueue(b, b->cfg, d_view, d_loc, (uint32_t)n, level, d_out, d_status, b->cap);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(b->cap, &graph);
        if (rc != RLFC_OK) {
            if (graph)
                cudaGraphDestroy(graph);
            return rc;
        }
        if (e != cudaSuccess)
            return cuda_fail(e, "batch graph capture");
        e = cudaGraphInstantiate(&b->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            b->exec = nullptr;
            return cuda_fail(e, "batch graph instantiate");
        }
        b->key = k;
    }
    cudaError_t e;
    {
        TraceScope trace_("batch_graph", st);
        e = cudaGraphLaunch(b->exec, st);
    }
    if (e != cudaSuccess)
        return cuda_fail(e, "batch graph launch");
    return RLFC_OK;
}

RLFC_API int rlfc_batch_autotune(rlfc_batch *b, const uint32_t *d_view, const uint32_t *d_loc, size_t n,
                                 uint8_t *d_out, uint8_t *d_status, void *cuda_stream,
                                 rlfc_batch_config *chosen)
{
    using namespace rlfc;
    int rc = check_args(b, d_view, d_loc, n, 0, d_out);
    if (rc != RLFC_OK)
        return rc;
    DeviceGuard g(b->device);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    rlfc_batch_config best = b->cfg;
    if (n > 0) {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        cudaError_t e = cudaEventCreate(&e0);
        if (e == cudaSuccess)
            e = cudaEventCreate(&e1);
        float best_ms = 1e30f;
        const uint32_t warps[3] = {4, 8, 16}, pops[2] = {1, 4};
        for (uint32_t wi = 0; wi < 3 && e == cudaSuccess && rc == RLFC_OK; wi++)
            for (uint32_t pi = 0; pi < 2 && e == cudaSuccess && rc == RLFC_OK; pi++)
                for (uint32_t stg = 0; stg < 3 && e == cudaSuccess && rc == RLFC_OK; stg++) {
                    if (stg == 2 && pi != 0)
                        continue;   // prefetching takes one location at a time
                    const rlfc_batch_config c{warps[wi], pops[pi], stg, b->cfg.graph};
                    if (!fits(b, c))
                        continue;
                    rc = enqueue(b, c, d_view, d_loc, (uint32_t)n, 0, d_out, d_status, st);   // warm-up
                    if (rc != RLFC_OK)
                        break;
                    e = cudaEventRecord(e0, st);
                    for (int rep = 0; rep < 3 && rc == RLFC_OK; rep++)
                        rc = enqueue(b, c, d_view, d_loc, (uint32_t)n, 0, d_out, d_status, st);
                    if (e == cudaSuccess)
                        e = cudaEventRecord(e1, st);
                    if (e == cudaSuccess)
                        e = cudaEventSynchronize(e1);
                    float ms = 0.f;
                    if (e == cudaSuccess)
                        e = cudaEventElapsedTime(&ms, e0, e1);
                    if (e == cudaSuccess && rc == RLFC_OK && ms < best_ms) {
                        best_ms = ms;
                        best = c;
                    }
                }
        if (e0)
            cudaEventDestroy(e0);
        if (e1)
            cudaEventDestroy(e1);
        if (rc != RLFC_OK)
            return rc;
        if (e != cudaSuccess)
            return cuda_fail(e, "batch autotune");
    }
    drop_graph(b);
    b->cfg = best;
    if (chosen)
        *chosen = best;
    return RLFC_OK;
}

RLFC_API void rlfc_batch_free(rlfc_batch *b)
{
    if (!b)
        return;
    rlfc::DeviceGuard g(b->device);
    // a decode still in flight may use the batch's buffers: let the device finish first
    cudaDeviceSynchronize();
    rlfc::drop_graph(b);
    if (b->cap)
        cudaStreamDestroy(b->cap);
    cudaFree(b->d_cnt);
    cudaFree(b->d_rank);
    cudaFree(b->d_sorted);
    cudaFree(b->d_sorted_view);
    delete b;
}

}  // extern "C"

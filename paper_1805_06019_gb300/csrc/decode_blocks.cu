// Random-access block decode, Algorithm 2 DecompressLFIBlock(ImgIdx, BlkIdx),
// for a batch of independent requests: one warp per request, using the
// warp-cooperative block decoder.  Out-of-range requests get a status byte
// and a zeroed block; nothing traps.
#include <cuda_runtime.h>

#include "warp_decode.cuh"

namespace rlfc {
namespace {

constexpr int kWarpsPerCta = 8;

__constant__ uint32_t c_modes[kNumModes] = RLFC_MODE_TABLE_INIT;

struct Args {
    StreamView sv;
    const uint32_t *req_view;
    const uint32_t *req_loc;
    uint8_t *out;
    uint8_t *status;
    uint32_t n;
    uint32_t aligned;   // output 4-byte aligned: store whole words
};

__global__ void __launch_bounds__(kWarpsPerCta * 32) decode_blocks_kernel(const Args a)
{
    __shared__ uint32_t s_mode[kNumModes];
    if (threadIdx.x < kNumModes)
        s_mode[threadIdx.x] = c_modes[threadIdx.x];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const uint32_t r = blockIdx.x * kWarpsPerCta + (threadIdx.x >> 5);
    if (r >= a.n)
        return;
    const uint32_t view = a.req_view[r], loc = a.req_loc[r];
    uint8_t *dst = a.out + (size_t)r * 48;
    const uint32_t bad = view >= a.sv.n_views ? (uint32_t)RLFC_REQ_BAD_VIEW
                                              : (loc >= a.sv.nloc ? (uint32_t)RLFC_REQ_BAD_LOCATION : 0u);
    if (a.status && lane == 0)
        a.status[r] = (uint8_t)bad;
    if (bad) {
        if (a.aligned) {
            if (lane < 12)
                reinterpret_cast<uint32_t *>(dst)[lane] = 0u;
        } else {
            for (int b = lane; b < 48; b += 32)
                dst[b] = 0;
        }
        return;
    }
    const uint32_t rgb = warp_decode_block(a.sv, s_mode, view, loc, lane);
    if (a.aligned) {
        // 48 bytes as 12 words: word w holds bytes 4w..4w+3, which start at
        // byte (4w) % 3 of pixel (4w) / 3 and end inside the next pixel
        const uint32_t p0 = (uint32_t)(lane * 4) / 3;
        const uint32_t lo = __shfl_sync(kFullMask, rgb, min(p0, 31u));
        const uint32_t hi = __shfl_sync(kFullMask, rgb, min(p0 + 1, 31u));
        if (lane < 12) {
            const uint32_t sh = (uint32_t)(lane * 4) % 3;   // first byte of the word inside pixel p0
            reinterpret_cast<uint32_t *>(dst)[lane] =
                __byte_perm(lo, hi, sh == 0 ? 0x4210u : (sh == 1 ? 0x5421u : 0x6542u));
        }
    } else if (lane < 16) {
        dst[3 * lane] = (uint8_t)rgb;
        dst[3 * lane + 1] = (uint8_t)(rgb >> 8);
        dst[3 * lane + 2] = (uint8_t)(rgb >> 16);
    }
}

// One thread per record: every stored block decoded, the largest
// |(min + u) * 2^(q + shift)| over the record, reduced per warp into *out.
__global__ void __launch_bounds__(256) block_magnitude_kernel(const uint32_t *records, const uint32_t *offsets,
                                                              uint32_t n_rec, uint32_t MW, uint32_t q,
                                                              uint32_t *out)
{
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t mx = 0;
    if (r < n_rec) {
        const uint32_t *rec = records + offsets[r];
        uint32_t P = 0;
        for (uint32_t w = 0; w < MW; w++)
            P += __popc(rec[w]);
        const uint32_t hdr0 = 32 * MW;
        uint32_t pos = hdr0 + kHdrBits * P;
        for (uint32_t h = 0; h < P; h++) {
            const BlockHeader hd = unpack_header(get_bits(rec, hdr0 + kHdrBits * h, kHdrBits));
            const uint32_t mode = c_modes[hd.mode];
            int32_t u[kVals];
            bise_decode16(rec, pos, mode, u);
            int32_t lo = u[0], hi = u[0];
#pragma unroll
            for (int v = 1; v < kVals; v++) {
                lo = min(lo, u[v]);
                hi = max(hi, u[v]);
            }
            const int32_t a = hd.min + lo, b = hd.min + hi;
            mx = max(mx, (uint32_t)max(abs(a), abs(b)) << (q + hd.shift));
            pos += mode_bits(mode);
        }
    }
    mx = __reduce_max_sync(kFullMask, mx);
    if ((threadIdx.x & 31) == 0)
        atomicMax(out, mx);
}

}  // namespace

int block_magnitude(const rlfc_stream *s, cudaStream_t st, uint32_t *mag)
{
    const uint32_t n_rec = 3 * s->info.nloc_x * s->info.nloc_y;
    uint32_t *d = nullptr;
    cudaError_t e = cudaMallocAsync(&d, 4, st);
    if (e != cudaSuccess)
        return cuda_fail(e, "block magnitude: allocation");
    if ((e = cudaMemsetAsync(d, 0, 4, st)) == cudaSuccess) {
        { rlfc::TraceScope trace_("block_magnitude_kernel", st); block_magnitude_kernel<<<(n_rec + 255) / 256, 256, 0, st>>>(s->d_records, s->d_offsets, n_rec, s->MW, s->info.q, d); }
        if ((e = cudaGetLastError()) == cudaSuccess && (e = cudaMemcpyAsync(mag, d, 4, cudaMemcpyDeviceToHost, st)) == cudaSuccess)
            e = cudaStreamSynchronize(st);
    }
    cudaFreeAsync(d, st);
    if (e != cudaSuccess)
        return cuda_fail(e, "block magnitude");
    return RLFC_OK;
}

int launch_decode_blocks(const rlfc_stream *s, const uint32_t *d_view, const uint32_t *d_loc, uint32_t n,
                         uint8_t *d_out, uint8_t *d_status, cudaStream_t st)
{
    Args a;
    a.sv.records = s->d_records;
    a.sv.offsets = s->d_offsets;
    a.sv.top = s->d_top;
    a.sv.view_anc = s->d_view_anc;
    a.sv.n_views = s->tab.n_views;
    a.sv.nloc = s->info.nloc_x * s->info.nloc_y;
    a.sv.nlx = s->info.nloc_x;
    a.sv.L = s->tab.L;
    a.sv.q = s->info.q;
    a.sv.MW = s->MW;
    a.sv.dbg = s->d_debug;
    a.req_view = d_view;
    a.req_loc = d_loc;
    a.out = d_out;
    a.status = d_status;
    a.n = n;
    a.aligned = ((uintptr_t)d_out & 3u) == 0;
    const uint32_t grid = (n + kWarpsPerCta - 1) / kWarpsPerCta;
    { rlfc::TraceScope trace_("decode_blocks_kernel", st); decode_blocks_kernel<<<grid, kWarpsPerCta * 32, 0, st>>>(a); }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_fail(e, "decode_blocks launch");
    return RLFC_OK;
}

}  // namespace rlfc

// GPU encoder, Algorithm 1 (CompressLFI):
//   RKV^0 <- YCoCg-R of the (edge-padded) views                 [ycocg_pad_kernel]
//   ComputeRKVTree: binomial-weighted cluster filter per level   [filter_kernel]
//   ComputeSRVTree: closed-loop residuals, pixel / block-energy
//                   thresholds, quantisation, reconstruction     [srv_kernel]
//   per (location, channel): BFS-ordered blocks -> mode, header,
//                   BISE payload                                 [record_size_kernel, record_pack_kernel]
//   stream = header : top RKVs (raw int16) : offsets : records   [host]
// Every rule is integer arithmetic (the filter is the binomial approximation
// of the Gaussian weighting, normalised by a power of two), so the stream is
// byte-identical to any other encoder that follows the same rules.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "rlfc_device.cuh"
#include "rlfc_internal.h"

namespace rlfc {
namespace {

// ranges of the 28 modes, ascending
__constant__ uint32_t c_rangeN[kNumModes] = {1,  2,  3,  4,   5,   6,   8,   10,  12,  16,  20,  24,  32,  40,
                                             48, 64, 80, 96, 128, 160, 192, 256, 320, 384, 512, 640, 768, 1024};
__constant__ uint32_t c_modes[kNumModes] = RLFC_MODE_TABLE_INIT;

#include "ks_device.cuh"

__global__ void ycocg_pad_kernel(const uint8_t *rgb, int16_t *x0, uint32_t n_views, uint32_t W, uint32_t H,
                                 uint32_t Wp, uint32_t Hp)
{
    const size_t plane = (size_t)Wp * Hp;
    const size_t total = plane * n_views;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const uint32_t view = (uint32_t)(i / plane);
        const uint32_t r = (uint32_t)(i - (size_t)view * plane);
        const uint32_t y = r / Wp, x = r - y * Wp;
        const uint32_t sx = min(x, W - 1), sy = min(y, H - 1);
        const uint8_t *p = rgb + (((size_t)view * H + sy) * W + sx) * 3;
        const int R = p[0], G = p[1], B = p[2];
        const int co = R - B;
        const int t = B + (co >> 1);
        const int cg = G - t;
        const int Y = t + (cg >> 1);
        int16_t *dst = x0 + (size_t)view * 3 * plane + r;
        dst[0] = (int16_t)Y;
        dst[plane] = (int16_t)co;
        dst[2 * plane] = (int16_t)cg;
    }
}

// One parent node per blockIdx.y: floor((sum w X + 2^(s-1)) / 2^s) over its
// members, with members/weights/shift given per parent.
__global__ void filter_kernel(const int16_t *child, int16_t *parent, const uint32_t *member_start,
                              const uint32_t *member_idx, const int64_t *member_w, const uint32_t *shift,
                              size_t npix)
{
    const uint32_t p = blockIdx.y;
    const uint32_t m0 = member_start[p], m1 = member_start[p + 1];
    const uint32_t s = shift[p];
    const int64_t half = s > 0 ? (int64_t)1 << (s - 1) : 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < npix; i += (size_t)gridDim.x * blockDim.x) {
        int64_t acc = 0;
        for (uint32_t m = m0; m < m1; m++)
            acc += member_w[m] * (int64_t)child[(size_t)member_idx[m] * npix + i];
        parent[(size_t)p * npix + i] = (int16_t)((acc + half) >> s);
    }
}

struct SrvArgs {
    int16_t *child;           // RKVs of level l-1; replaced by the quantised SRV
    const int16_t *rec_par;   // reconstruction of level l
    int16_t *rec_child;       // reconstruction of level l-1 (null for level 0)
    const uint32_t *parent;   // parent index of each child node
    uint8_t *present;         // [child node][3][nloc]
    uint8_t *kmode;           // [child node][3][nloc]: k | s << 5 of a stored block
    const uint8_t *leaf_modes;   // level 0 only, may be null: given k | s << 5, 0xFF = search
    int16_t *leaf_resid;      // level 0 only, may be null: residuals after the pixel threshold
    uint8_t *leaf_label;      // level 0 only, may be null: search result, 0xFF = not kept
    int *error;
    uint32_t n_child, nlx, nloc, Wp, Hp;
    int32_t tau_p, tau_b;
    uint32_t q;
    uint32_t mode_space, lam_q8;
    int32_t tau_err;
};

// (shift, mode) search: ks_device.cuh, included above with these tables in scope

// Eq. 3 with the thresholds and quantisation of Section 3.2, one thread per
// (child node, channel, block location).
__global__ void srv_kernel(const SrvArgs a)
{
    const size_t plane = (size_t)a.Wp * a.Hp;
    const size_t total = (size_t)a.n_child * 3 * a.nloc;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const uint32_t node = (uint32_t)(i / (3 * (size_t)a.nloc));
        const uint32_t rem = (uint32_t)(i - (size_t)node * 3 * a.nloc);
        const uint32_t c = rem / a.nloc, loc = rem - c * a.nloc;
        const uint32_t bx = loc % a.nlx, by = loc / a.nlx;
        const uint32_t par = a.parent[node];
        int16_t *xc = a.child + ((size_t)node * 3 + c) * plane;
        const int16_t *xp = a.rec_par + ((size_t)par * 3 + c) * plane;
        int r[kVals];
        int energy = 0;
#pragma unroll
        for (int k = 0; k < kVals; k++) {
            const size_t at = (size_t)(by * 4 + k / 4) * a.Wp + bx * 4 + k % 4;
            int v = xc[at] - xp[at];
            if (abs(v) < a.tau_p)
                v = 0;
            r[k] = v;
            energy += abs(v);
        }
        bool keep = energy > 0 && energy >= a.tau_b;
        const size_t bi = ((size_t)node * 3 + c) * a.nloc + loc;
        if (a.leaf_resid) {
#pragma unroll
            for (int k = 0; k < kVals; k++)
                a.leaf_resid[bi * kVals + k] = (int16_t)r[k];
        }
        if (a.leaf_label) {
            uint32_t lk = 0, ls = 0;
            a.leaf_label[bi] = keep && ks_search(r, a.q, a.tau_err, a.lam_q8, lk, ls) ? (uint8_t)(lk | ls << 5)
                                                                                     : (uint8_t)0xFF;
        }
        uint32_t ks_k = 0, ks_s = 0;
        if (keep && a.mode_space) {
            bool have = false;
            if (a.leaf_modes && a.leaf_modes[bi] != 0xFF) {
                // a given mode is used when it is a candidate
                const uint32_t gk = a.leaf_modes[bi] & 31u, gs = a.leaf_modes[bi] >> 5;
                long long cost;
                if (ks_cost(r, a.q, gs, gk, a.tau_err, a.lam_q8, cost)) {
                    ks_k = gk;
                    ks_s = gs;
                    have = true;
                }
            }
            if (!have && !ks_search(r, a.q, a.tau_err, a.lam_q8, ks_k, ks_s))
                atomicExch(a.error, 3);
        }
        const uint32_t t = a.q + ks_s;
        const int half = t > 0 ? 1 << (t - 1) : 0;
        bool nonzero = false;
        int mn = 0, mx = 0;
#pragma unroll
        for (int k = 0; k < kVals; k++) {
            const int qm = (abs(r[k]) + half) >> t;
            r[k] = keep ? (r[k] < 0 ? -qm : qm) : 0;
            nonzero |= r[k] != 0;
            mn = k == 0 ? r[k] : min(mn, r[k]);
            mx = k == 0 ? r[k] : max(mx, r[k]);
        }
        keep = keep && nonzero;
        if (keep && !a.mode_space) {
            // the plain method: the smallest range that holds the span
            while (ks_k < kNumModes - 1 && (int)c_rangeN[ks_k] < mx - mn + 1)
                ks_k++;
        }
        a.present[bi] = keep ? 1 : 0;
        a.kmode[bi] = keep ? (uint8_t)(ks_k | ks_s << 5) : 0;
        int16_t *rc = a.rec_child ? a.rec_child + ((size_t)node * 3 + c) * plane : nullptr;
#pragma unroll
        for (int k = 0; k < kVals; k++) {
            const size_t at = (size_t)(by * 4 + k / 4) * a.Wp + bx * 4 + k % 4;
            const int qv = keep ? r[k] : 0;
            if (rc)
                rc[at] = (int16_t)(xp[at] + qv * (1 << t));
            xc[at] = (int16_t)qv;
        }
    }
}

struct RecArgs {
    const int16_t *const *srv;   // per level < L-1: quantised SRV images
    const uint8_t *const *present;
    const uint8_t *const *kmode;  // per level < L-1: k | s << 5 of each stored block
    const uint32_t *bfs_level;   // [S]
    const uint32_t *bfs_node;    // [S]
    uint32_t S, MW, nlx, nloc, Wp, Hp;
    uint32_t *words;             // record_size: per-record word count; record_pack: the records
    const uint32_t *offsets;     // record_pack only
    int *error;
};

__device__ __forceinline__ void load_block(const RecArgs &a, uint32_t pos, uint32_t c, uint32_t loc,
                                           int v[kVals], bool &present, uint32_t &km)
{
    const uint32_t lv = a.bfs_level[pos], nd = a.bfs_node[pos];
    present = a.present[lv][((size_t)nd * 3 + c) * a.nloc + loc] != 0;
    if (!present)
        return;
    km = a.kmode[lv][((size_t)nd * 3 + c) * a.nloc + loc];
    const size_t plane = (size_t)a.Wp * a.Hp;
    const int16_t *img = a.srv[lv] + ((size_t)nd * 3 + c) * plane;
    const uint32_t bx = loc % a.nlx, by = loc / a.nlx;
#pragma unroll
    for (int k = 0; k < kVals; k++)
        v[k] = img[(size_t)(by * 4 + k / 4) * a.Wp + bx * 4 + k % 4];
}

__global__ void record_size_kernel(const RecArgs a)
{
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= 3 * a.nloc)
        return;
    const uint32_t loc = r / 3, c = r - 3 * loc;
    uint32_t bits = 32 * a.MW;
    for (uint32_t pos = 0; pos < a.S; pos++) {
        int v[kVals];
        bool present;
        uint32_t km = 0;
        load_block(a, pos, c, loc, v, present, km);
        if (!present)
            continue;
        int mn = v[0], mx = v[0];
#pragma unroll
        for (int k = 1; k < kVals; k++) {
            mn = min(mn, v[k]);
            mx = max(mx, v[k]);
        }
        if ((int)c_rangeN[km & 31u] < mx - mn + 1 || mn < -1024 || mn > 1023)
            atomicExch(a.error, 1);
        bits += kHdrBits + mode_bits(c_modes[km & 31u]);
    }
    a.words[r] = (bits + 31) / 32;
}

struct BitWriter {
    uint32_t *out;
    uint64_t acc;
    uint32_t n;
    __device__ __forceinline__ void put(uint32_t v, uint32_t width)
    {
        acc |= (uint64_t)v << n;
        n += width;
        if (n >= 32) {
            *out++ = (uint32_t)acc;
            acc >>= 32;
            n -= 32;
        }
    }
    __device__ __forceinline__ void flush()
    {
        if (n > 0)
            *out++ = (uint32_t)acc;
        acc = 0;
        n = 0;
    }
};

__global__ void record_pack_kernel(const RecArgs a)
{
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= 3 * a.nloc)
        return;
    const uint32_t loc = r / 3, c = r - 3 * loc;
    uint32_t *rec = a.words + a.offsets[r];
    const uint32_t nwords = a.offsets[r + 1] - a.offsets[r];
    // presence mask
    for (uint32_t m = 0; m < a.MW; m++) {
        uint32_t w = 0;
        for (uint32_t b = 0; b < 32 && m * 32 + b < a.S; b++) {
            const uint32_t pos = m * 32 + b;
            const uint32_t lv = a.bfs_level[pos], nd = a.bfs_node[pos];
            if (a.present[lv][((size_t)nd * 3 + c) * a.nloc + loc])
                w |= 1u << b;
        }
        rec[m] = w;
    }
    BitWriter bw{rec + a.MW, 0, 0};
    // headers: mode 5 | shift 2 | min 11
    for (uint32_t pos = 0; pos < a.S; pos++) {
        int v[kVals];
        bool present;
        uint32_t km = 0;
        load_block(a, pos, c, loc, v, present, km);
        if (!present)
            continue;
        int mn = v[0];
#pragma unroll
        for (int k = 1; k < kVals; k++)
            mn = min(mn, v[k]);
        bw.put((km & 31u) | ((km >> 5) << 5) | (((uint32_t)mn & 0x7FFu) << 7), kHdrBits);
    }
    // payloads: digit words, then the low bits
    for (uint32_t pos = 0; pos < a.S; pos++) {
        int v[kVals];
        bool present;
        uint32_t km = 0;
        load_block(a, pos, c, loc, v, present, km);
        if (!present)
            continue;
        int mn = v[0];
#pragma unroll
        for (int k = 1; k < kVals; k++)
            mn = min(mn, v[k]);
        const uint32_t m = c_modes[km & 31u];
        const uint32_t b = mode_b(m), kind = mode_kind(m);
        uint32_t u[kVals];
#pragma unroll
        for (int k = 0; k < kVals; k++)
            u[k] = (uint32_t)(v[k] - mn);
        if (kind == 1) {
#pragma unroll
            for (int g = 0; g < 4; g++) {
                uint32_t word = 0, scale = 1;
#pragma unroll
                for (int e = 0; e < 5; e++) {
                    const int k = 5 * g + e;
                    if (k < kVals) {
                        word += (u[k] >> b) * scale;
                        scale *= 3;
                    }
                }
                bw.put(word, g < 3 ? 8u : 2u);
            }
        } else if (kind == 2) {
#pragma unroll
            for (int g = 0; g < 6; g++) {
                uint32_t word = 0, scale = 1;
#pragma unroll
                for (int e = 0; e < 3; e++) {
                    const int k = 3 * g + e;
                    if (k < kVals) {
                        word += (u[k] >> b) * scale;
                        scale *= 5;
                    }
                }
                bw.put(word, g < 5 ? 7u : 3u);
            }
        }
#pragma unroll
        for (int k = 0; k < kVals; k++)
            bw.put(u[k] & ((1u << b) - 1u), b);
    }
    bw.flush();
    if ((uint32_t)(bw.out - rec) != nwords)
        atomicExch(a.error, 2);
}

int tile_count(uint32_t G, uint32_t c) { return (int)((G + c - 1) / c); }

struct DevBuf {
    std::vector<void *> ptrs;
    uint8_t *arena = nullptr;   // when set, buffers are carved from this caller-provided block
    size_t arena_size = 0, arena_used = 0;
    ~DevBuf()
    {
        for (void *p : ptrs)
            cudaFree(p);
    }
    template <typename T>
    cudaError_t alloc(T **p, size_t count)
    {
        if (arena) {
            const size_t at = (arena_used + 255) & ~size_t(255);
            const size_t bytes = count * sizeof(T) + 16;
            if (at + bytes > arena_size)
                return cudaErrorMemoryAllocation;
            *p = reinterpret_cast<T *>(arena + at);
            arena_used = at + bytes;
            return cudaSuccess;
        }
        cudaError_t e = cudaMalloc((void **)p, count * sizeof(T) + 16);
        if (e == cudaSuccess)
            ptrs.push_back((void *)*p);
        return e;
    }
};

void put32(std::vector<uint8_t> &b, size_t at, uint32_t v)
{
    b[at] = (uint8_t)v;
    b[at + 1] = (uint8_t)(v >> 8);
    b[at + 2] = (uint8_t)(v >> 16);
    b[at + 3] = (uint8_t)(v >> 24);
}

size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

}  // namespace

// Upper bound of the device scratch encode_gpu carves for these parameters
// (every buffer rounded up to 256 bytes, records at their largest possible
// size); 0 when the parameters are invalid.
size_t encode_scratch_bound(const rlfc_enc_params *p)
{
    if (!p || p->B != 4 || p->U < 1 || p->V < 1 || (uint64_t)p->U * p->V > 16383 || p->W < 1 || p->H < 1 ||
        p->W > 65536 || p->H > 65536 || p->L < 2 || p->L > (uint32_t)kMaxLevels)
        return 0;
    const uint32_t L = p->L;
    std::vector<uint64_t> cnt(L);
    uint64_t Gu = p->U, Gv = p->V;
    cnt[0] = Gu * Gv;
    for (uint32_t l = 1; l < L; l++) {
        if (p->c[l] < 1)
            return 0;
        Gu = (Gu + p->c[l] - 1) / p->c[l];
        Gv = (Gv + p->c[l] - 1) / p->c[l];
        cnt[l] = Gu * Gv;
    }
    const uint64_t Wp = (p->W + 3) / 4 * 4, Hp = (p->H + 3) / 4 * 4, nloc = (Wp / 4) * (Hp / 4);
    const uint64_t npix = 3 * Wp * Hp;
    uint64_t S = 0;
    for (uint32_t l = 0; l + 1 < L; l++)
        S += cnt[l];
    uint64_t total = 0;
    auto add = [&](uint64_t bytes) { total += ((bytes + 16) + 255) / 256 * 256; };
    for (uint32_t l = 0; l < L; l++) {
        add(2 * npix * cnt[l]);
        if (l >= 1 && l + 1 < L)
            add(2 * npix * cnt[l]);
        if (l + 1 < L)
            add(cnt[l] * 3 * nloc);
        if (l + 1 < L)
            add(cnt[l] * 3 * nloc);
    }
    add(sizeof(int));
    add(sizeof(void *) * L);
    for (uint32_t l = 1; l < L; l++) {
        add(4 * (cnt[l] + 1));
        add(4 * cnt[l - 1]);
        add(4 * cnt[l]);
        add(8 * cnt[l - 1]);
        add(4 * cnt[l - 1]);
    }
    add(4 * S);
    add(4 * S);
    add(4 * 3 * nloc);
    add(4 * (3 * nloc + 1));
    add(sizeof(int));
    add(sizeof(void *) * L);
    add(sizeof(void *) * L);
    const uint64_t MW = (S + 31) / 32;
    add(4 * (3 * nloc * (MW + (S * (kHdrBits + 160) + 31) / 32) + 1));
    return (size_t)total;
}

int encode_gpu(const rlfc_enc_params *p, const uint8_t *d_rgb, cudaStream_t st, std::vector<uint8_t> &out,
               uint8_t *arena, size_t arena_size, const uint8_t *d_leaf_modes, int16_t *d_leaf_resid,
               uint8_t *d_leaf_label)
{
    if (p->B != 4) {
        set_error("the GPU encoder writes 4x4 blocks only");
        return RLFC_E_UNSUPPORTED;
    }
    if (p->U < 1 || p->V < 1 || (uint64_t)p->U * p->V > 16383 || p->W < 1 || p->H < 1 || p->W > 65536 ||
        p->H > 65536 || p->L < 2 || p->L > (uint32_t)kMaxLevels || p->tau_p < 0 || p->tau_b < 0 || p->q > 7 ||
        p->mode_space > 1 || p->tau_err < 0) {
        set_error("encoder parameters out of range");
        return RLFC_E_INVALID_ARG;
    }
    const uint32_t L = p->L;
    for (uint32_t l = 1; l < L; l++)
        if (p->c[l] < 1) {
            set_error("cluster side must be >= 1");
            return RLFC_E_INVALID_ARG;
        }
    // tree shape (Eq. 1 reading): uniform tiling per level
    std::vector<uint32_t> Gu(L), Gv(L), cnt(L);
    Gu[0] = p->U;
    Gv[0] = p->V;
    for (uint32_t l = 1; l < L; l++) {
        Gu[l] = tile_count(Gu[l - 1], p->c[l]);
        Gv[l] = tile_count(Gv[l - 1], p->c[l]);
    }
    for (uint32_t l = 0; l < L; l++)
        cnt[l] = Gu[l] * Gv[l];
    std::vector<std::vector<uint32_t>> parent(L);
    // tile a of k covering G nodes: [floor(aG/k), floor((a+1)G/k))
    auto tile_of = [](uint32_t x, uint32_t G, uint32_t k) {
        uint32_t a = 0;
        while (!((uint64_t)(a + 1) * G / k > x))
            a++;
        return a;
    };
    for (uint32_t l = 0; l + 1 < L; l++) {
        parent[l].resize(cnt[l]);
        for (uint32_t y = 0; y < Gv[l]; y++)
            for (uint32_t x = 0; x < Gu[l]; x++)
                parent[l][y * Gu[l] + x] = tile_of(y, Gv[l], Gv[l + 1]) * Gu[l + 1] + tile_of(x, Gu[l], Gu[l + 1]);
    }
    Tables tab;
    if (build_tables(L, cnt, parent, tab) != 0 || tab.S >= 16384) {
        set_error("tree too large");
        return RLFC_E_RANGE;
    }
    const uint32_t W = p->W, H = p->H, Wp = (W + 3) / 4 * 4, Hp = (H + 3) / 4 * 4;
    const uint32_t nlx = Wp / 4, nly = Hp / 4, nloc = nlx * nly;
    const size_t plane = (size_t)Wp * Hp, npix = 3 * plane;

    DevBuf buf;
    buf.arena = arena;
    buf.arena_size = arena_size;
    cudaError_t e;
    std::vector<int16_t *> img(L, nullptr), rec(L, nullptr);
    std::vector<uint8_t *> present(L, nullptr), kmode(L, nullptr);
    for (uint32_t l = 0; l < L; l++) {
        if ((e = buf.alloc(&img[l], npix * cnt[l])) != cudaSuccess)
            return cuda_fail(e, "encoder allocation");
        if (l >= 1 && l + 1 < L && (e = buf.alloc(&rec[l], npix * cnt[l])) != cudaSuccess)
            return cuda_fail(e, "encoder allocation");
        if (l + 1 < L && (e = buf.alloc(&present[l], (size_t)cnt[l] * 3 * nloc)) != cudaSuccess)
            return cuda_fail(e, "encoder allocation");
        if (l + 1 < L && (e = buf.alloc(&kmode[l], (size_t)cnt[l] * 3 * nloc)) != cudaSuccess)
            return cuda_fail(e, "encoder allocation");
    }
    int *d_err;
    if ((e = buf.alloc(&d_err, 1)) != cudaSuccess)
        return cuda_fail(e, "encoder allocation");
    cudaMemsetAsync(d_err, 0, sizeof(int), st);
    rec[L - 1] = img[L - 1];
    const int threads = 256;
    auto grid_for = [](size_t n) { return (unsigned)std::min<size_t>((n + 255) / 256, 152 * 64); };

    { rlfc::TraceScope trace_("ycocg_pad_kernel", st); ycocg_pad_kernel<<<grid_for(plane * cnt[0]), threads, 0, st>>>(d_rgb, img[0], cnt[0], W, H, Wp, Hp); }

    // bottom-up filter
    for (uint32_t l = 1; l < L; l++) {
        std::vector<uint32_t> mstart(1, 0), midx, shift;
        std::vector<int64_t> mw;
        const uint32_t ku = Gu[l], kv = Gv[l];
        for (uint32_t b = 0; b < kv; b++)
            for (uint32_t a2 = 0; a2 < ku; a2++) {
                const uint32_t x0 = (uint64_t)a2 * Gu[l - 1] / ku, x1 = (uint64_t)(a2 + 1) * Gu[l - 1] / ku;
                const uint32_t y0 = (uint64_t)b * Gv[l - 1] / kv, y1 = (uint64_t)(b + 1) * Gv[l - 1] / kv;
                const uint32_t mu = x1 - x0, mv = y1 - y0;
                // Pascal's triangle rows mu-1 and mv-1
                std::vector<int64_t> ru(mu, 1), rv(mv, 1);
                for (uint32_t i = 1; i + 1 < mu; i++)
                    ru[i] = ru[i - 1] * (mu - i) / i;
                for (uint32_t i = 1; i + 1 < mv; i++)
                    rv[i] = rv[i - 1] * (mv - i) / i;
                for (uint32_t y = y0; y < y1; y++)
                    for (uint32_t x = x0; x < x1; x++) {
                        midx.push_back(y * Gu[l - 1] + x);
                        mw.push_back(ru[x - x0] * rv[y - y0]);
                    }
                mstart.push_back((uint32_t)midx.size());
                shift.push_back((mu - 1) + (mv - 1));
                if ((mu - 1) + (mv - 1) > 40) {
                    set_error("cluster too large");
                    return RLFC_E_RANGE;
                }
            }
        uint32_t *d_ms, *d_mi, *d_sh;
        int64_t *d_mw;
        if ((e = buf.alloc(&d_ms, mstart.size())) != cudaSuccess || (e = buf.alloc(&d_mi, midx.size())) != cudaSuccess ||
            (e = buf.alloc(&d_sh, shift.size())) != cudaSuccess || (e = buf.alloc(&d_mw, mw.size())) != cudaSuccess)
            return cuda_fail(e, "encoder allocation");
        cudaMemcpyAsync(d_ms, mstart.data(), 4 * mstart.size(), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(d_mi, midx.data(), 4 * midx.size(), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(d_sh, shift.data(), 4 * shift.size(), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(d_mw, mw.data(), 8 * mw.size(), cudaMemcpyHostToDevice, st);
        dim3 grid((unsigned)std::min<size_t>((npix + 255) / 256, 4096), cnt[l]);
        { rlfc::TraceScope trace_("filter_kernel", st); filter_kernel<<<grid, threads, 0, st>>>(img[l - 1], img[l], d_ms, d_mi, d_mw, d_sh, npix); }
        // keep the host vectors alive until the copies are done
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess)
            return cuda_fail(e, "encoder filter");
    }

    // top-down residuals (closed loop)
    for (uint32_t l = L - 1; l >= 1; l--) {
        uint32_t *d_par;
        if ((e = buf.alloc(&d_par, cnt[l - 1])) != cudaSuccess)
            return cuda_fail(e, "encoder allocation");
        cudaMemcpyAsync(d_par, parent[l - 1].data(), 4ull * cnt[l - 1], cudaMemcpyHostToDevice, st);
        SrvArgs s;
        s.child = img[l - 1];
        s.rec_par = rec[l];
        s.rec_child = (l - 1 >= 1) ? rec[l - 1] : nullptr;
        s.parent = d_par;
        s.present = present[l - 1];
        s.kmode = kmode[l - 1];
        s.leaf_modes = l == 1 ? d_leaf_modes : nullptr;
        s.leaf_resid = l == 1 ? d_leaf_resid : nullptr;
        s.leaf_label = l == 1 ? d_leaf_label : nullptr;
        s.error = d_err;
        s.mode_space = p->mode_space;
        s.lam_q8 = p->lam_q8;
        s.tau_err = p->tau_err;
        s.n_child = cnt[l - 1];
        s.nlx = nlx;
        s.nloc = nloc;
        s.Wp = Wp;
        s.Hp = Hp;
        s.tau_p = p->tau_p;
        s.tau_b = p->tau_b;
        s.q = p->q;
        { rlfc::TraceScope trace_("srv_kernel", st); srv_kernel<<<grid_for((size_t)cnt[l - 1] * 3 * nloc), threads, 0, st>>>(s); }
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess)
            return cuda_fail(e, "encoder residuals");
    }

    // BFS tables for the record kernels
    std::vector<uint32_t> bfs_level(tab.S), bfs_node(tab.S);
    for (uint32_t pos = 0; pos < tab.S; pos++)
        bfs_level[pos] = node_level(tab.node_info[pos]);
    // node index of every BFS position: every node is an ancestor of some view
    for (uint32_t v = 0; v < cnt[0]; v++) {
        uint32_t a2 = v;
        for (uint32_t l = 0; l + 1 < L; l++) {
            bfs_node[tab.view_anc[(size_t)v * kMaxLevels + l]] = a2;
            a2 = parent[l][a2];
        }
    }
    const uint32_t S = tab.S, MW = (S + 31) / 32;
    uint32_t *d_bl, *d_bn, *d_words_n, *d_off, *d_rec;
    const int16_t **d_srv;
    const uint8_t **d_pres, **d_km;
    if ((e = buf.alloc(&d_bl, S)) != cudaSuccess || (e = buf.alloc(&d_bn, S)) != cudaSuccess ||
        (e = buf.alloc(&d_words_n, 3ull * nloc)) != cudaSuccess || (e = buf.alloc(&d_off, 3ull * nloc + 1)) != cudaSuccess ||
        (e = buf.alloc(&d_srv, L)) != cudaSuccess || (e = buf.alloc(&d_pres, L)) != cudaSuccess ||
        (e = buf.alloc(&d_km, L)) != cudaSuccess)
        return cuda_fail(e, "encoder allocation");
    std::vector<const int16_t *> srv_ptrs(img.begin(), img.end());
    std::vector<const uint8_t *> pres_ptrs(present.begin(), present.end()), km_ptrs(kmode.begin(), kmode.end());
    cudaMemcpyAsync(d_bl, bfs_level.data(), 4ull * S, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(d_bn, bfs_node.data(), 4ull * S, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(d_srv, srv_ptrs.data(), sizeof(void *) * L, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(d_pres, pres_ptrs.data(), sizeof(void *) * L, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(d_km, km_ptrs.data(), sizeof(void *) * L, cudaMemcpyHostToDevice, st);
    RecArgs ra;
    ra.srv = d_srv;
    ra.present = d_pres;
    ra.kmode = d_km;
    ra.bfs_level = d_bl;
    ra.bfs_node = d_bn;
    ra.S = S;
    ra.MW = MW;
    ra.nlx = nlx;
    ra.nloc = nloc;
    ra.Wp = Wp;
    ra.Hp = Hp;
    ra.words = d_words_n;
    ra.offsets = nullptr;
    ra.error = d_err;
    { rlfc::TraceScope trace_("record_size_kernel", st); record_size_kernel<<<(3 * nloc + 127) / 128, 128, 0, st>>>(ra); }
    std::vector<uint32_t> words(3ull * nloc), offsets(3ull * nloc + 1);
    int h_err = 0;
    cudaMemcpyAsync(words.data(), d_words_n, 4ull * 3 * nloc, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_fail(e, "encoder record sizes");
    if (h_err) {
        set_error(h_err == 3 ? "a residual block has no (mode, shift) candidate"
                             : "a residual block's range does not fit the 28 BISE modes");
        return RLFC_E_RANGE;
    }
    uint64_t total = 0;
    for (size_t i = 0; i < words.size(); i++) {
        offsets[i] = (uint32_t)total;
        total += words[i];
    }
    offsets.back() = (uint32_t)total;
    if (total >= (1ull << 32) - 16) {
        set_error("stream larger than 16 GiB");
        return RLFC_E_RANGE;
    }
    if ((e = buf.alloc(&d_rec, total + 1)) != cudaSuccess)
        return cuda_fail(e, "encoder allocation");
    cudaMemcpyAsync(d_off, offsets.data(), 4ull * offsets.size(), cudaMemcpyHostToDevice, st);
    ra.words = d_rec;
    ra.offsets = d_off;
    { rlfc::TraceScope trace_("record_pack_kernel", st); record_pack_kernel<<<(3 * nloc + 127) / 128, 128, 0, st>>>(ra); }

    // assemble the stream
    const size_t hdr_end = 64 + 8ull * L + 4ull * S;
    const size_t off_top = align16(hdr_end);
    const size_t top_bytes = 2ull * cnt[L - 1] * npix;
    const size_t off_offsets = align16(off_top + top_bytes);
    const size_t off_records = align16(off_offsets + 4ull * offsets.size());
    out.assign(off_records + 4ull * total, 0);
    const uint32_t hdr[15] = {0x43464C52u, 1u, p->U, p->V, W, H, 4u, L, p->q, cnt[L - 1], S,
                              (uint32_t)off_top, (uint32_t)off_offsets, (uint32_t)off_records, (uint32_t)total};
    for (int i = 0; i < 15; i++)
        put32(out, 4 * i, hdr[i]);
    size_t at = 64;
    for (uint32_t l = 0; l < L; l++, at += 8) {
        put32(out, at, Gu[l]);
        put32(out, at + 4, Gv[l]);
    }
    for (uint32_t l = 0; l + 1 < L; l++)
        for (uint32_t i = 0; i < cnt[l]; i++, at += 4)
            put32(out, at, parent[l][i]);
    cudaMemcpyAsync(out.data() + off_top, img[L - 1], top_bytes, cudaMemcpyDeviceToHost, st);
    for (size_t i = 0; i < offsets.size(); i++)
        put32(out, off_offsets + 4 * i, offsets[i]);
    cudaMemcpyAsync(out.data() + off_records, d_rec, 4ull * total, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_fail(e, "encoder packing");
    if (h_err) {
        set_error("record packing disagreed with the sizing pass");
        return RLFC_E_CUDA;
    }
    return RLFC_OK;
}

}  // namespace rlfc

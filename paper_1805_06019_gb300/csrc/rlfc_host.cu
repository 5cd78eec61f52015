// Host side of the RLFC library: the C ABI, the stream parser / validator and
// the decoder initialisation of Algorithm 2 (read the top RKVs, the block
// offsets and the SRV stream, and rebuild the BFS numbering, Section 3.5).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "rlfc_internal.h"

namespace rlfc {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

int cuda_fail(cudaError_t e, const char *what)
{
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? RLFC_E_OOM : RLFC_E_CUDA;
}

namespace {

constexpr uint32_t kMagic = 0x43464C52u;  // "RLFC"

uint32_t rd32(const uint8_t *p) { return p[0] | (p[1] << 8) | (p[2] << 16) | ((uint32_t)p[3] << 24); }
uint64_t align16(uint64_t x) { return (x + 15) & ~uint64_t(15); }

// payload bits of a 16-value block in mode k (bits / trits / quints), as the
// ascending range table 1 2 3 4 5 6 8 10 12 16 ... 768 1024 implies
uint32_t payload_bits16(uint32_t k)
{
    if (k < 3)
        return k == 2 ? 26u : 16u * k;
    const uint32_t g = (k - 3) / 3, r = (k - 3) % 3;
    if (r == 0)
        return 16u * (g + 2);       // 2^(g+2)
    if (r == 1)
        return 16u * g + 38u;       // 5 * 2^g
    return 16u * (g + 1) + 26u;     // 3 * 2^(g+1)
}

// the range N of mode k (1 2 3 4 5 6 8 10 12 16 ... 768 1024)
uint32_t range16(uint32_t k)
{
    if (k < 3)
        return k + 1;
    const uint32_t g = (k - 3) / 3, r = (k - 3) % 3;
    return r == 0 ? 4u << g : (r == 1 ? 5u << g : 6u << g);
}

// Largest |Y|, |Co|, |Cg| the GPU kernels accept: they hold reconstructions
// and the inverse YCoCg-R intermediates (up to 3M + 2) as 16-bit values with
// a bias of 2^14.
constexpr uint64_t kMaxMagnitude = 5460;

}  // namespace

// BFS numbering of the SRV nodes (Section 3.4): start from every top node in
// index order, visit children in increasing node index.  Fills the per-position
// node table and every view's ancestors.
int build_tables(uint32_t L, const std::vector<uint32_t> &cnt,
                 const std::vector<std::vector<uint32_t>> &parent, Tables &t)
{
    std::vector<std::vector<std::vector<uint32_t>>> children(L);
    for (uint32_t l = 0; l + 1 < L; l++) {
        children[l + 1].assign(cnt[l + 1], {});
        for (uint32_t i = 0; i < cnt[l]; i++)
            children[l + 1][parent[l][i]].push_back(i);
    }
    uint32_t S = 0;
    for (uint32_t l = 0; l + 1 < L; l++)
        S += cnt[l];
    std::vector<std::vector<uint32_t>> pos(L);
    for (uint32_t l = 0; l < L; l++)
        pos[l].assign(cnt[l], 0xFFFFFFFFu);
    std::vector<std::pair<uint32_t, uint32_t>> queue;
    queue.reserve(S + cnt[L - 1]);
    for (uint32_t i = 0; i < cnt[L - 1]; i++)
        queue.push_back({L - 1, i});
    t.L = L;
    t.S = S;
    t.n_top = cnt[L - 1];
    t.n_views = cnt[0];
    t.node_info.assign(S, 0);
    uint32_t next = 0;
    for (size_t h = 0; h < queue.size(); h++) {
        const uint32_t lv = queue[h].first, nd = queue[h].second;
        if (lv + 1 < L) {
            pos[lv][nd] = next;
            const uint32_t par = parent[lv][nd];
            const uint32_t pref = (lv + 2 == L) ? par : pos[lv + 1][par];
            t.node_info[next] = lv | (pref << 4) | ((lv == 0 ? nd : 0u) << 18);
            next++;
        }
        if (lv > 0)
            for (uint32_t ch : children[lv][nd])
                queue.push_back({lv - 1, ch});
    }
    if (next != S)
        return -1;
    t.n_int = S - cnt[0];   // BFS lists all levels >= 1 before the views
    t.view_anc.assign((size_t)t.n_views * kMaxLevels, 0);
    for (uint32_t v = 0; v < t.n_views; v++) {
        uint32_t a = v;
        for (uint32_t l = 0; l + 1 < L; l++) {
            t.view_anc[(size_t)v * kMaxLevels + l] = pos[l][a];
            a = parent[l][a];
        }
        t.view_anc[(size_t)v * kMaxLevels + L - 1] = a;
    }
    return 0;
}

namespace {

int fmt(const std::string &m)
{
    set_error("stream format: " + m);
    return RLFC_E_FORMAT;
}

struct Parsed {
    uint32_t U, V, W, H, B, L, q, n_top, S;
    uint64_t off_top, off_offsets, off_records, record_words;
    uint32_t Wp, Hp, nlx, nly, nloc, MW, max_record_words, max_strip_words, max_present, max_strip_present;
    std::vector<uint32_t> present;   // stored blocks of each record
    uint64_t max_top_mag, max_block_mag;   // largest |top value| and bound on |block value|
    Tables tab;
};

int parse(const uint8_t *p, size_t n, Parsed &ps)
{
    if (n < 64)
        return fmt("shorter than the 64-byte header");
    if (rd32(p) != kMagic)
        return fmt("bad magic");
    if (rd32(p + 4) != 1)
        return fmt("unknown version");
    ps.U = rd32(p + 8); ps.V = rd32(p + 12); ps.W = rd32(p + 16); ps.H = rd32(p + 20);
    ps.B = rd32(p + 24); ps.L = rd32(p + 28); ps.q = rd32(p + 32);
    ps.n_top = rd32(p + 36); ps.S = rd32(p + 40);
    ps.off_top = rd32(p + 44); ps.off_offsets = rd32(p + 48); ps.off_records = rd32(p + 52);
    ps.record_words = rd32(p + 56);
    if (ps.U < 1 || ps.V < 1 || ps.U > 4096 || ps.V > 4096 || (uint64_t)ps.U * ps.V > 16383)
        return fmt("view grid out of range");
    if (ps.W < 1 || ps.H < 1 || ps.W > 65536 || ps.H > 65536)
        return fmt("view size out of range");
    if (ps.B < 1 || ps.B > 8 || ps.L < 2 || ps.L > (uint32_t)kMaxLevels || ps.q > 7)
        return fmt("block size, level count or quantisation out of range");
    const uint32_t L = ps.L;
    if (64 + 8ull * L > n)
        return fmt("truncated level table");
    std::vector<uint32_t> Gu(L), Gv(L), cnt(L);
    uint64_t srv_nodes = 0;
    for (uint32_t l = 0; l < L; l++) {
        Gu[l] = rd32(p + 64 + 8 * l);
        Gv[l] = rd32(p + 68 + 8 * l);
        if (Gu[l] < 1 || Gv[l] < 1 || Gu[l] > 4096 || Gv[l] > 4096)
            return fmt("level grid out of range");
        cnt[l] = Gu[l] * Gv[l];
        if (l + 1 < L)
            srv_nodes += cnt[l];
    }
    if (Gu[0] != ps.U || Gv[0] != ps.V)
        return fmt("level 0 is not the view grid");
    if (cnt[L - 1] != ps.n_top || srv_nodes != ps.S || ps.S >= 16384 || ps.n_top >= 16384)
        return fmt("node counts disagree with the level grids");
    const uint64_t hdr_end = 64 + 8ull * L + 4ull * ps.S;
    if (hdr_end > n)
        return fmt("truncated parent table");
    // parent tables and children lists (children in increasing node index)
    std::vector<std::vector<uint32_t>> parent(L);
    uint64_t at = 64 + 8ull * L;
    for (uint32_t l = 0; l + 1 < L; l++) {
        parent[l].resize(cnt[l]);
        for (uint32_t i = 0; i < cnt[l]; i++, at += 4) {
            uint32_t par = rd32(p + at);
            if (par >= cnt[l + 1])
                return fmt("parent index out of range");
            parent[l][i] = par;
        }
    }
    if (build_tables(L, cnt, parent, ps.tab) != 0)
        return fmt("tree is not connected");
    // sections
    ps.Wp = (ps.W + ps.B - 1) / ps.B * ps.B;
    ps.Hp = (ps.H + ps.B - 1) / ps.B * ps.B;
    ps.nlx = ps.Wp / ps.B;
    ps.nly = ps.Hp / ps.B;
    ps.nloc = ps.nlx * ps.nly;
    const uint64_t top_bytes = 2ull * ps.n_top * 3 * ps.Wp * ps.Hp;
    const uint64_t noff = 3ull * ps.nloc + 1;
    if (ps.off_top != align16(hdr_end) || ps.off_offsets != align16(ps.off_top + top_bytes) ||
        ps.off_records != align16(ps.off_offsets + 4 * noff) ||
        ps.off_records + 4 * ps.record_words != n)
        return fmt("section offsets or total size inconsistent");
    // offsets and records
    ps.MW = (ps.S + 31) / 32;
    ps.max_record_words = 0;
    ps.max_present = 0;
    ps.present.assign(noff - 1, 0u);
    ps.max_block_mag = 0;
    ps.max_top_mag = 0;
    for (uint64_t i = 0; i < top_bytes / 2; i++) {
        const int32_t v = (int16_t)(uint16_t)(p[ps.off_top + 2 * i] | (p[ps.off_top + 2 * i + 1] << 8));
        ps.max_top_mag = std::max<uint64_t>(ps.max_top_mag, (uint64_t)(v < 0 ? -v : v));
    }
    const uint8_t *off = p + ps.off_offsets;
    const uint8_t *rec = p + ps.off_records;
    if (rd32(off) != 0 || rd32(off + 4 * (noff - 1)) != ps.record_words)
        return fmt("first or last offset wrong");
    for (uint64_t r = 0; r + 1 < noff; r++) {
        const uint32_t w0 = rd32(off + 4 * r), w1 = rd32(off + 4 * r + 4);
        if (w1 < w0 || w1 > ps.record_words)
            return fmt("offsets not increasing");
        const uint32_t words = w1 - w0;
        ps.max_record_words = std::max(ps.max_record_words, words);
        if (words < ps.MW)
            return fmt("record shorter than its presence mask");
        const uint8_t *rp = rec + 4ull * w0;
        uint32_t P = 0;
        for (uint32_t m = 0; m < ps.MW; m++) {
            uint32_t w = rd32(rp + 4 * m);
            if (m == ps.MW - 1 && (ps.S & 31))
                if (w >> (ps.S & 31))
                    return fmt("presence bits beyond the last node");
            P += __builtin_popcount(w);
        }
        ps.max_present = std::max(ps.max_present, P);
        ps.present[r] = P;
        uint64_t bits = 32ull * ps.MW + 18ull * P;
        if (bits > 32ull * words)
            return fmt("block headers run past the record");
        if (ps.B == 4) {
            for (uint32_t h = 0; h < P; h++) {
                const uint64_t hp = 32ull * ps.MW + 18ull * h;
                const uint64_t wi = hp >> 5;
                uint64_t win = rd32(rp + 4 * wi);
                if (wi + 1 < words)
                    win |= (uint64_t)rd32(rp + 4 * (wi + 1)) << 32;
                const uint32_t hdr = (uint32_t)(win >> (hp & 31)) & 0x3FFFFu;
                const uint32_t k = hdr & 31u;
                if (k >= 28)
                    return fmt("block mode out of range");
                bits += payload_bits16(k);
                // |(min + u) * 2^(q + shift)| for u in [0, N)
                const int64_t mn = ((int32_t)(hdr << 14)) >> 21;
                const int64_t hi = mn + (int64_t)range16(k) - 1;
                const uint64_t mag = (uint64_t)std::max(mn < 0 ? -mn : mn, hi < 0 ? -hi : hi)
                                     << (ps.q + ((hdr >> 5) & 3u));
                ps.max_block_mag = std::max(ps.max_block_mag, mag);
            }
            if ((bits + 31) / 32 != words)
                return fmt("record length disagrees with its blocks");
        }
    }
    // the longest run of records of kDecodeStrip consecutive locations of a
    // row (the full decode stages one such run per CTA)
    ps.max_strip_words = 0;
    ps.max_strip_present = 0;
    for (uint32_t y = 0; y < ps.nly; y++)
        for (uint32_t x0 = 0; x0 < ps.nlx; x0 += kDecodeStrip) {
            const uint32_t b0 = y * ps.nlx + x0, b1 = y * ps.nlx + std::min(x0 + kDecodeStrip, ps.nlx);
            ps.max_strip_words = std::max(ps.max_strip_words, rd32(off + 12ull * b1) - rd32(off + 12ull * b0));
            uint32_t sp = 0;
            for (uint64_t r = 3ull * b0; r < 3ull * b1; r++)
                sp += ps.present[r];
            ps.max_strip_present = std::max(ps.max_strip_present, sp);
        }
    if (ps.B != 4) {
        set_error("the GPU kernels decode 4x4 blocks only");
        return RLFC_E_UNSUPPORTED;
    }
    if (ps.max_top_mag > kMaxMagnitude) {
        set_error("reconstructed values can leave the 16-bit range of the GPU kernels");
        return RLFC_E_UNSUPPORTED;
    }
    return RLFC_OK;
}

void free_device(rlfc_stream *s)
{
    cudaFree(s->d_records);
    cudaFree(s->d_offsets);
    cudaFree(s->d_top);
    cudaFree(s->d_node_info);
    cudaFree(s->d_view_anc);
    cudaFree(s->d_debug);
    s->d_debug = nullptr;
    s->d_records = nullptr;
    s->d_offsets = nullptr;
    s->d_top = nullptr;
    s->d_node_info = nullptr;
    s->d_view_anc = nullptr;
}

int load(const uint8_t *bytes, size_t nbytes, cudaStream_t st, rlfc_stream **out)
{
    Parsed ps;
    int rc = parse(bytes, nbytes, ps);
    if (rc != RLFC_OK)
        return rc;
    rlfc_stream *s = new rlfc_stream();
    cudaGetDevice(&s->device);
    s->tab = std::move(ps.tab);
    s->MW = ps.MW;
    s->record_words = ps.record_words;
    s->max_record_words = ps.max_record_words;
    s->max_strip_words = ps.max_strip_words;
    s->max_present = ps.max_present;
    s->max_strip_present = ps.max_strip_present;
    rlfc_info &in = s->info;
    in.U = ps.U; in.V = ps.V; in.W = ps.W; in.H = ps.H; in.B = ps.B; in.L = ps.L; in.q = ps.q;
    in.n_top = ps.n_top; in.S = ps.S; in.Wp = ps.Wp; in.Hp = ps.Hp;
    in.nloc_x = ps.nlx; in.nloc_y = ps.nly;
    in.stream_bytes = nbytes;
    in.record_bytes = 4ull * ps.record_words;
    in.top_bytes = 2ull * ps.n_top * 3 * ps.Wp * ps.Hp;

    // top RKVs, block-major: [top][loc][channel][16]
    const uint32_t nloc = ps.nloc;
    std::vector<int16_t> top((size_t)ps.n_top * nloc * 48);
    const uint8_t *tp = bytes + ps.off_top;
    for (uint32_t t = 0; t < ps.n_top; t++)
        for (uint32_t c = 0; c < 3; c++)
            for (uint32_t y = 0; y < ps.Hp; y++)
                for (uint32_t x = 0; x < ps.Wp; x++) {
                    const size_t src = (((size_t)t * 3 + c) * ps.Hp + y) * ps.Wp + x;
                    const uint32_t loc = (y / 4) * ps.nlx + x / 4;
                    const uint32_t v = (y % 4) * 4 + x % 4;
                    int16_t val;
                    std::memcpy(&val, tp + 2 * src, 2);
                    top[((size_t)t * nloc + loc) * 48 + c * 16 + v] = val;
                }
    const size_t rec_bytes = 4ull * (ps.record_words + kPadWords);
    const size_t off_bytes = 4ull * (3ull * nloc + 1);
    const size_t top_bytes = top.size() * 2;
    const size_t ni_bytes = 4ull * s->tab.S;
    const size_t va_bytes = 4ull * s->tab.view_anc.size();
    cudaError_t e;
    if ((e = cudaMalloc(&s->d_records, rec_bytes)) != cudaSuccess ||
        (e = cudaMalloc(&s->d_offsets, off_bytes)) != cudaSuccess ||
        (e = cudaMalloc(&s->d_top, top_bytes)) != cudaSuccess ||
        (e = cudaMalloc(&s->d_node_info, ni_bytes)) != cudaSuccess ||
        (e = cudaMalloc(&s->d_view_anc, va_bytes)) != cudaSuccess
#ifdef RLFC_DEBUG
        || (e = cudaMalloc(&s->d_debug, 4)) != cudaSuccess || (e = cudaMemsetAsync(s->d_debug, 0, 4, st)) != cudaSuccess
#endif
    ) {
        free_device(s);
        delete s;
        return cuda_fail(e, "device allocation for the stream");
    }
    in.device_bytes = rec_bytes + off_bytes + top_bytes + ni_bytes + va_bytes;
    if ((e = cudaMemsetAsync(s->d_records, 0, rec_bytes, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(s->d_records, bytes + ps.off_records, 4ull * ps.record_words,
                             cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(s->d_offsets, bytes + ps.off_offsets, off_bytes,
                             cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(s->d_top, top.data(), top_bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(s->d_node_info, s->tab.node_info.data(), ni_bytes,
                             cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(s->d_view_anc, s->tab.view_anc.data(), va_bytes,
                             cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess) {
        free_device(s);
        delete s;
        return cuda_fail(e, "uploading the stream");
    }
    // the headers bound every block value; where that bound is too loose for
    // the 16-bit range, decode every block once and take the exact bound
    if (ps.max_top_mag + (uint64_t)(ps.L - 1) * ps.max_block_mag > kMaxMagnitude) {
        uint32_t mag = 0;
        const int rc = block_magnitude(s, st, &mag);
        if (rc != RLFC_OK || ps.max_top_mag + (uint64_t)(ps.L - 1) * mag > kMaxMagnitude) {
            free_device(s);
            delete s;
            if (rc != RLFC_OK)
                return rc;
            set_error("reconstructed values can leave the 16-bit range of the GPU kernels");
            return RLFC_E_UNSUPPORTED;
        }
    }
    *out = s;
    return RLFC_OK;
}

}  // namespace
}  // namespace rlfc

using namespace rlfc;

extern "C" {

int rlfc_load_stream(const void *host_bytes, size_t nbytes, void *cuda_stream, rlfc_stream **out)
{
    if (!host_bytes || !out) {
        set_error("null argument");
        return RLFC_E_INVALID_ARG;
    }
    *out = nullptr;
    try {
        return load(static_cast<const uint8_t *>(host_bytes), nbytes, (cudaStream_t)cuda_stream, out);
    } catch (const std::bad_alloc &) {
        set_error("host allocation failed");
        return RLFC_E_OOM;
    }
}

int rlfc_stream_info(const rlfc_stream *s, rlfc_info *out)
{
    if (!s || !out) {
        set_error("null argument");
        return RLFC_E_INVALID_ARG;
    }
    *out = s->info;
    return RLFC_OK;
}

void rlfc_free_stream(rlfc_stream *s)
{
    if (!s)
        return;
    DeviceGuard g(s->device);
    // kernels still in flight may read the stream (a caller that drops its
    // handle right after an asynchronous call): let the device finish first
    cudaDeviceSynchronize();
    free_device(s);
    delete s;
}

int rlfc_debug_flags(const rlfc_stream *s, uint32_t *flags, int reset)
{
    if (!s || !flags) {
        set_error("null argument");
        return RLFC_E_INVALID_ARG;
    }
    *flags = 0;
    if (!s->d_debug) {
        set_error("the library was built without RLFC_DEBUG");
        return RLFC_E_UNSUPPORTED;
    }
    DeviceGuard g(s->device);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess)
        e = cudaMemcpy(flags, s->d_debug, 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && reset)
        e = cudaMemset(s->d_debug, 0, 4);
    if (e != cudaSuccess)
        return cuda_fail(e, "reading the debug flags");
    return RLFC_OK;
}

int rlfc_decode_all(const rlfc_stream *s, uint8_t *d_out, void *cuda_stream)
{
    if (!s || !d_out) {
        set_error("null argument");
        return RLFC_E_INVALID_ARG;
    }
    DeviceGuard g(s->device);
    return launch_decode_all(s, d_out, (cudaStream_t)cuda_stream);
}

int rlfc_decode_blocks(const rlfc_stream *s, const uint32_t *d_view, const uint32_t *d_loc,
                       size_t n, uint8_t *d_out, uint8_t *d_status, void *cuda_stream)
{
    if (!s) {
        set_error("null stream");
        return RLFC_E_INVALID_ARG;
    }
    if (n == 0)
        return RLFC_OK;
    if (!d_view || !d_loc || !d_out) {
        set_error("null argument");
        return RLFC_E_INVALID_ARG;
    }
    if (n >= (size_t(1) << 31)) {
        set_error("at most 2^31 - 1 requests per call");
        return RLFC_E_RANGE;
    }
    DeviceGuard g(s->device);
    return launch_decode_blocks(s, d_view, d_loc, (uint32_t)n, d_out, d_status,
                                (cudaStream_t)cuda_stream);
}

static int render_common(const rlfc_stream *s, const float *d_uv, const float *d_disp, uint32_t out_w,
                         uint32_t out_h, size_t n, float *d_out, uint8_t *d_out8, void *cuda_stream)
{
    if (!s) {
        set_error("null stream");
        return RLFC_E_INVALID_ARG;
    }
    if (n == 0)
        return RLFC_OK;
    if (!d_uv || !d_disp || (!d_out && !d_out8) || out_w == 0 || out_h == 0) {
        set_error("null argument or empty output size");
        return RLFC_E_INVALID_ARG;
    }
    if (n >= 65536 || out_w > 32768 || out_h > 32768) {
        set_error("at most 65535 views of 32768 x 32768 per call");
        return RLFC_E_RANGE;
    }
    DeviceGuard g(s->device);
    return launch_render(s, d_uv, d_disp, out_w, out_h, (uint32_t)n, d_out, (cudaStream_t)cuda_stream, d_out8);
}

int rlfc_render_views(const rlfc_stream *s, const float *d_uv, const float *d_disp,
                      uint32_t out_w, uint32_t out_h, size_t n, float *d_out, void *cuda_stream)
{
    return render_common(s, d_uv, d_disp, out_w, out_h, n, d_out, nullptr, cuda_stream);
}

int rlfc_render_views_u8(const rlfc_stream *s, const float *d_uv, const float *d_disp,
                         uint32_t out_w, uint32_t out_h, size_t n, uint8_t *d_out, void *cuda_stream)
{
    return render_common(s, d_uv, d_disp, out_w, out_h, n, nullptr, d_out, cuda_stream);
}

int rlfc_encode(const rlfc_enc_params *p, const uint8_t *d_rgb, void *cuda_stream, void **host_out,
                size_t *nbytes)
{
    return rlfc_encode_ex(p, d_rgb, nullptr, nullptr, nullptr, cuda_stream, host_out, nbytes);
}

int rlfc_encode_ex(const rlfc_enc_params *p, const uint8_t *d_rgb, const uint8_t *d_leaf_modes,
                   int16_t *d_leaf_resid, uint8_t *d_leaf_label, void *cuda_stream, void **host_out,
                   size_t *nbytes)
{
    if (!p || !d_rgb || !host_out || !nbytes) {
        set_error("null argument");
        return RLFC_E_INVALID_ARG;
    }
    *host_out = nullptr;
    *nbytes = 0;
    try {
        std::vector<uint8_t> out;
        int rc = encode_gpu(p, d_rgb, (cudaStream_t)cuda_stream, out, nullptr, 0, d_leaf_modes, d_leaf_resid,
                            d_leaf_label);
        if (rc != RLFC_OK)
            return rc;
        void *buf = std::malloc(out.size());
        if (!buf) {
            set_error("host allocation failed");
            return RLFC_E_OOM;
        }
        std::memcpy(buf, out.data(), out.size());
        *host_out = buf;
        *nbytes = out.size();
        return RLFC_OK;
    } catch (const std::bad_alloc &) {
        set_error("host allocation failed");
        return RLFC_E_OOM;
    }
}

void rlfc_free_host(void *p) { std::free(p); }

const char *rlfc_strerror(int code)
{
    switch (code) {
    case RLFC_OK: return "ok";
    case RLFC_E_INVALID_ARG: return "invalid argument";
    case RLFC_E_FORMAT: return "corrupt or truncated stream";
    case RLFC_E_UNSUPPORTED: return "unsupported stream parameters";
    case RLFC_E_CUDA: return "CUDA error";
    case RLFC_E_OOM: return "out of memory";
    case RLFC_E_RANGE: return "size out of range";
    case RLFC_E_TIMEOUT: return "device wait timed out";
    default: return "unknown status";
    }
}

const char *rlfc_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

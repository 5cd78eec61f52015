// Internal state of a loaded RLFC stream and the kernel launchers.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/rlfc.h"

namespace rlfc {

constexpr int kMaxLevels = 8;
constexpr uint32_t kDecodeStrip = 8;   // block locations per CTA of the full decode
constexpr int kPadWords = 16;  // zero words after the records (decoder and staging over-read)

// Per BFS position: level (bits 0..3), parent reference (bits 4..17: the top
// RKV index when the parent is the top level, else the parent's BFS
// position), view index for level-0 nodes (bits 18..31).
__host__ __device__ inline uint32_t node_level(uint32_t w) { return w & 15u; }
__host__ __device__ inline uint32_t node_parent(uint32_t w) { return (w >> 4) & 0x3FFFu; }
__host__ __device__ inline uint32_t node_view(uint32_t w) { return w >> 18; }

struct Tables {
    uint32_t L = 0, S = 0, n_top = 0, n_int = 0, n_views = 0;
    std::vector<uint32_t> node_info;  // [S]
    std::vector<uint32_t> view_anc;   // [n_views][kMaxLevels]: BFS position of the ancestor at
                                      // levels 0..L-2, the top index at L-1
};

}  // namespace rlfc

struct rlfc_stream {
    rlfc_info info{};
    int device = 0;
    rlfc::Tables tab;
    uint32_t MW = 0;            // mask words per record
    uint64_t record_words = 0;
    uint32_t max_record_words = 0;
    uint32_t max_strip_words = 0;    // records of kDecodeStrip consecutive locations of a row
    uint32_t max_present = 0;        // most stored blocks in one record
    uint32_t max_strip_present = 0;  // most stored blocks in the records of kDecodeStrip consecutive locations of a row
    // device buffers
    uint32_t *d_records = nullptr;   // record_words + kPadWords
    uint32_t *d_offsets = nullptr;   // 3 * nloc + 1
    int16_t *d_top = nullptr;        // [n_top][nloc][3][16], block-major YCoCg-R
    uint32_t *d_node_info = nullptr; // [S]
    uint32_t *d_view_anc = nullptr;  // [n_views][kMaxLevels]
    uint32_t *d_debug = nullptr;     // debug builds: the bounds checks' flag word (rlfc_debug_flags)
};

namespace rlfc {

void set_error(const std::string &msg);

// Records CUDA events around the launches made during its lifetime when
// tracing is on (rlfc_trace_enable); the name must be a string literal.
class TraceScope {
public:
    TraceScope(const char *name, cudaStream_t st);
    ~TraceScope();
    TraceScope(const TraceScope &) = delete;
    TraceScope &operator=(const TraceScope &) = delete;

private:
    const char *name_;
    cudaStream_t st_;
    cudaEvent_t a_ = nullptr, b_ = nullptr;
};

// Makes `dev` current for its lifetime and restores the previous device.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev)
            cudaSetDevice(dev);
        else
            prev = -1;
    }
    ~DeviceGuard()
    {
        if (prev >= 0)
            cudaSetDevice(prev);
    }
};

int build_tables(uint32_t L, const std::vector<uint32_t> &cnt,
                 const std::vector<std::vector<uint32_t>> &parent, Tables &t);
int cuda_fail(cudaError_t e, const char *what);

int launch_decode_all(const rlfc_stream *s, uint8_t *d_out, cudaStream_t st);
// every view the mask marks (all when null), as packed RGB words [view][H][W]
// Packed RGB words of the views `needed` marks, view v into slot slot_of[v]
// of d_out ([slot][H][W], n_slots slots); with needed null, every view v into
// slot v.
int launch_decode_packed(const rlfc_stream *s, uint32_t *d_out, const uint8_t *needed, const uint32_t *slot_of,
                         uint32_t n_slots, cudaStream_t st);
// Largest |value| of any stored block of the stream, decoded (synchronous).
int block_magnitude(const rlfc_stream *s, cudaStream_t st, uint32_t *mag);
int launch_decode_blocks(const rlfc_stream *s, const uint32_t *d_view, const uint32_t *d_loc,
                         uint32_t n, uint8_t *d_out, uint8_t *d_status, cudaStream_t st);
// d_out8: when set, 8-bit RGB output instead of d_out
int launch_render_native(const rlfc_stream *s, const float *d_uv, const float *d_disp, uint32_t n,
                         float *d_out, cudaStream_t st, uint8_t *d_out8 = nullptr);
int launch_render(const rlfc_stream *s, const float *d_uv, const float *d_disp, uint32_t out_w,
                  uint32_t out_h, uint32_t n, float *d_out, cudaStream_t st, uint8_t *d_out8 = nullptr);
// arena: when given, every device buffer of the encoder is carved from it
// (arena_size bytes) instead of being allocated
// d_leaf_modes / d_leaf_resid / d_leaf_label: optional level-0 mode input and
// training-data outputs (see rlfc_encode_ex)
int encode_gpu(const rlfc_enc_params *p, const uint8_t *d_rgb, cudaStream_t st,
               std::vector<uint8_t> &out, uint8_t *arena = nullptr, size_t arena_size = 0,
               const uint8_t *d_leaf_modes = nullptr, int16_t *d_leaf_resid = nullptr,
               uint8_t *d_leaf_label = nullptr);
size_t encode_scratch_bound(const rlfc_enc_params *p);

}  // namespace rlfc

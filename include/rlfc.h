/*
 * rlfc.h -- C ABI of the GB300 RLFC library (librlfc.so).
 *
 * RLFC (Pratapa & Manocha, I3D 2019) stores a light field as a tree: a few
 * top-level representative key views (RKVs) plus sparse residual views (SRVs)
 * cut into blocks and packed with bounded integer sequence encoding (BISE).
 * Any block of any view can be decoded on its own ("random access", Section
 * 3.5).  This library decodes such streams on one GPU and renders new views
 * from them.
 *
 * Conventions for every call:
 *  - Pointers named d_* are device pointers owned by the caller; the library
 *    never frees them.  Host pointers are only read during the call.
 *  - `cuda_stream` is a cudaStream_t passed as void* (NULL = the legacy
 *    default stream).  Compute calls only enqueue work on it and return
 *    without synchronising; their outputs are valid once the stream reaches
 *    that point.
 *  - Every call returns RLFC_OK (0) or one of the RLFC_E_* codes.  Arguments
 *    the host can check are checked before anything is enqueued; on error
 *    nothing is written.  rlfc_strerror() turns a code into text and
 *    rlfc_last_error() gives the detail of the most recent failure on the
 *    calling thread.
 *  - A loaded rlfc_stream is immutable: calls on different CUDA streams may
 *    run concurrently against the same rlfc_stream.
 *  - Device code never traps: a request the host cannot check (out-of-range
 *    view or location inside a device array) gets a non-zero status byte and
 *    a zeroed output block.
 *
 * Stream format v1 (all fields little-endian):
 *   bytes 0..63   "RLFC", version 1, U, V, W, H, B, L, q, n_top, S, off_top,
 *                 off_offsets, off_records, record_words, 0 (uint32 each)
 *   then          per level l = 0..L-1 its node grid (Gu_l, Gv_l); then for
 *                 every node of levels 0..L-2 (row-major per level) the index of
 *                 its parent one level up
 *   off_top       the n_top top-level RKVs, int16 YCoCg-R, [n_top][3][Hp][Wp]
 *   off_offsets   3 * nloc + 1 uint32: start word of record (loc, channel) in
 *                 the record section, then the total word count
 *   off_records   the records, block locations row-major, channels Y, Co, Cg.
 * The SRV nodes (all tree nodes below the top level) are numbered by a
 * breadth-first search that starts from the top nodes in index order and
 * visits children in increasing node index.  A record holds ceil(S/32) mask
 * words (bit p set = SRV node p stores a block here), then one 18-bit header
 * per stored block in BFS order (mode 0..27 in bits 0..4, extra shift in bits
 * 5..6, block minimum as 11-bit two's complement in bits 7..17), then the
 * blocks' BISE payloads in the same order, zero-padded to a 32-bit word.  Bit
 * p of a record is bit p % 32 of its word p / 32.  Mode k codes values in
 * [0, N_k) with N_k ascending over {1,2,3,4,5,6,8,10,12,16,...,768,1024}
 * (2^b, 3*2^b, 5*2^b); a payload is the digit words first (trits: five per
 * 8-bit base-3 word, quints: three per 7-bit base-5 word, a short last group
 * taking ceil(8j/5) or ceil(7j/3) bits) and then each value's b low bits.  A
 * stored value contributes (min + u) * 2^(q + shift) to its pixel.
 */
#ifndef RLFC_H
#define RLFC_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define RLFC_API __attribute__((visibility("default")))
#else
#define RLFC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

enum rlfc_status {
    RLFC_OK = 0,
    RLFC_E_INVALID_ARG = 1,  /* null pointer, zero size where not allowed, bad enum */
    RLFC_E_FORMAT = 2,       /* stream bytes are corrupt or truncated */
    RLFC_E_UNSUPPORTED = 3,  /* valid stream the kernels do not handle (e.g. B != 4) */
    RLFC_E_CUDA = 4,         /* a CUDA runtime call failed */
    RLFC_E_OOM = 5,          /* device or host allocation failed */
    RLFC_E_RANGE = 6,        /* a size is beyond what the call supports */
    RLFC_E_TIMEOUT = 7       /* a bounded device wait gave up */
};

/* Per-request status bytes written by rlfc_decode_blocks. */
enum rlfc_request_status {
    RLFC_REQ_OK = 0,
    RLFC_REQ_BAD_VIEW = 1,
    RLFC_REQ_BAD_LOCATION = 2
};

typedef struct rlfc_stream rlfc_stream;  /* opaque, library-owned */

typedef struct {
    uint32_t U, V;           /* camera grid: views are indexed j * U + i */
    uint32_t W, H;           /* view size in pixels */
    uint32_t B;              /* block side (pixels) */
    uint32_t L;              /* tree levels, level 0 = the views */
    uint32_t q;              /* global quantisation shift */
    uint32_t n_top;          /* top-level RKVs */
    uint32_t S;              /* SRV nodes (tree nodes below the top level) */
    uint32_t Wp, Hp;         /* W, H rounded up to a multiple of B */
    uint32_t nloc_x, nloc_y; /* block locations per row / column */
    uint64_t stream_bytes;   /* size of the stream that was loaded */
    uint64_t record_bytes;   /* SRV record section */
    uint64_t top_bytes;      /* top RKV section */
    uint64_t device_bytes;   /* device memory held by the loaded stream */
} rlfc_info;

/*
 * Algorithm 2, initialisation (Section 3.5): parse and validate a stream held
 * in host memory (nbytes bytes), rebuild the BFS numbering of the tree, and
 * copy the top RKVs, the block offsets and the SRV records to the current
 * CUDA device.  Every record is checked on the host (mask, modes, lengths)
 * so that kernels never read past a record.  The copy is done on
 * `cuda_stream` and the call returns after it completes, so host_bytes may be
 * freed right away.  *out receives a handle to release with rlfc_free_stream.
 * Errors: RLFC_E_INVALID_ARG, RLFC_E_FORMAT, RLFC_E_OOM, RLFC_E_CUDA, and
 * RLFC_E_UNSUPPORTED for blocks other than 4 x 4 or when the largest |top
 * value| plus (L - 1) times the largest |block value| exceeds 5460 (the
 * kernels hold reconstructions in 16 bits; streams encoded from 8-bit views
 * stay far below).  The block bound comes from the headers, or, where that
 * bound is too loose, from decoding every block once on the device.
 */
RLFC_API int rlfc_load_stream(const void *host_bytes, size_t nbytes, void *cuda_stream,
                     rlfc_stream **out);

/* Shape and sizes of a loaded stream. */
RLFC_API int rlfc_stream_info(const rlfc_stream *s, rlfc_info *out);

/* Release a loaded stream and its device memory.  It first waits for the
 * stream's device to finish all queued work (cudaDeviceSynchronize), so work
 * that reads the stream may still be in flight when it is called. */
RLFC_API void rlfc_free_stream(rlfc_stream *s);

/*
 * Algorithm 2 for every block of every view (the "decode all blocks"
 * workload): d_out receives U*V*H*W*3 bytes, views in index order, each H rows
 * of W RGB pixels (padding cropped).  Errors: RLFC_E_INVALID_ARG,
 * RLFC_E_UNSUPPORTED, RLFC_E_CUDA.
 */
RLFC_API int rlfc_decode_all(const rlfc_stream *s, uint8_t *d_out, void *cuda_stream);

/*
 * Algorithm 2, DecompressLFIBlock(ImgIdx, BlkIdx), for n independent random
 * requests: request r decodes block location d_loc[r] (row-major, 0 <=
 * loc < nloc_x * nloc_y) of view d_view[r] (0 <= view < U * V).  d_out
 * receives n * B*B*3 bytes, request-major, each block B rows of B RGB pixels
 * (padding included).  d_status (n bytes, may be NULL) receives an
 * rlfc_request_status per request; a bad request gets a zeroed block.
 * n = 0 is a no-op.  Errors: RLFC_E_INVALID_ARG, RLFC_E_RANGE (n >= 2^31),
 * RLFC_E_UNSUPPORTED, RLFC_E_CUDA.
 */
RLFC_API int rlfc_decode_blocks(const rlfc_stream *s, const uint32_t *d_view, const uint32_t *d_loc,
                       size_t n, uint8_t *d_out, uint8_t *d_status, void *cuda_stream);

/*
 * Section 3.6: render n new views by quadrilinear interpolation of the
 * decoded light field, decoding the needed blocks on demand from the
 * compressed stream.  View r is seen from the continuous camera position
 * (d_uv[2r], d_uv[2r+1]) on the U x V grid (clamped to [0,U-1] x [0,V-1]) with
 * the focal plane at disparity d_disp[r] pixels per view.  Output pixel
 * (x, y) of an out_w x out_h image follows the ray through
 * s = (x + 0.5) W / out_w - 0.5, t = (y + 0.5) H / out_h - 0.5; in neighbour
 * view (i, j) it samples (s + d (i - u), t + d (j - v)) bilinearly with
 * clamp-to-edge, and the four views are blended bilinearly in (u, v).
 * d_out receives n * out_h * out_w * 3 floats (RGB in [0, 1]), view-major.
 * At native size a call of four or more cameras first decodes the neighbour
 * views they need into a transient device buffer (stream-ordered
 * allocation on cuda_stream, released before the call's work completes:
 * 4 * W * H bytes per needed view, at most min(views, 4n) of them); if that
 * allocation fails the call decodes on demand instead.  Results do not
 * depend on the path or on the other views of the call.
 * Errors: RLFC_E_INVALID_ARG, RLFC_E_RANGE, RLFC_E_UNSUPPORTED, RLFC_E_CUDA.
 */
RLFC_API int rlfc_render_views(const rlfc_stream *s, const float *d_uv, const float *d_disp,
                      uint32_t out_w, uint32_t out_h, size_t n, float *d_out,
                      void *cuda_stream);

/*
 * rlfc_render_views with 8-bit output, the displayable form of the same
 * views: d_out receives n * out_h * out_w * 3 bytes, each
 * floor(clamp(v, 0, 1) * 255 + 0.5) of the float value v that
 * rlfc_render_views computes (the product and the sum rounded separately in
 * FP32).  Errors: as rlfc_render_views.
 */
RLFC_API int rlfc_render_views_u8(const rlfc_stream *s, const float *d_uv, const float *d_disp,
                                  uint32_t out_w, uint32_t out_h, size_t n, uint8_t *d_out,
                                  void *cuda_stream);

/*
 * Batched random access (the paper's DecompressLFIBlock of Algorithm 2 for
 * many requests at once, Section 3.5, which notes that blocks decode in
 * parallel).  A batch object groups the requests of one call by block
 * location (a counting sort on the GPU), then a persistent kernel takes
 * locations from an atomic work queue: a warp parses a location's three
 * channel records once (presence mask ranks, header lengths, payload offsets)
 * and decodes the stored ancestor blocks of every request at that location,
 * so the record gather is shared by all of them.  The results are the same
 * bytes as rlfc_decode_blocks.
 *
 * Progressive decode (Section 3.6: stopping the traversal at a coarser
 * level returns the filtered views): with level l > 0 a request returns the
 * reconstruction of its view's level-l ancestor, i.e. the top RKV plus the
 * residuals of levels L-2 down to l, converted to RGB and clamped;
 * level L-1 returns the top RKV alone, level 0 the view itself.
 */
typedef struct rlfc_batch rlfc_batch;   /* opaque, library-owned */

typedef struct {
    uint32_t warps_per_cta;   /* 4, 8 or 16 */
    uint32_t locs_per_pop;    /* locations a warp takes from the queue at once, 1..64 */
    uint32_t stage;           /* 0: read a location's records through L1; 1: copy them to
                                 shared memory before parsing; 2: copy the next location's
                                 records (cp.async) while serving the current one (with
                                 locs_per_pop 1); records too long for the buffers are read
                                 through L1 */
    uint32_t graph;           /* 1: replay the call as a captured CUDA graph */
} rlfc_batch_config;

/*
 * Create a batch object for up to max_requests requests per call on stream s
 * (which must outlive it).  It allocates its device scratch (about
 * 12 B per request + 4 B per block location) on s's device, plus a private
 * CUDA stream used only to capture graphs.  The default configuration is
 * {8, 1, 0, 1}.  Errors: RLFC_E_INVALID_ARG, RLFC_E_RANGE (max_requests >=
 * 2^31), RLFC_E_UNSUPPORTED (records too large for the decoder's shared
 * memory), RLFC_E_OOM, RLFC_E_CUDA.
 */
RLFC_API int rlfc_batch_create(const rlfc_stream *s, size_t max_requests, rlfc_batch **out);

/* Set / read the configuration (validated; a new one drops the cached graph). */
RLFC_API int rlfc_batch_set_config(rlfc_batch *b, const rlfc_batch_config *cfg);
RLFC_API int rlfc_batch_get_config(const rlfc_batch *b, rlfc_batch_config *cfg);

/*
 * Decode n requests (view d_view[r], location d_loc[r], as for
 * rlfc_decode_blocks) at tree level `level` (0 = the views, up to L-1) into
 * d_out (n * 48 bytes, request-major, 16 RGB pixels row-major per block) and
 * d_status (n bytes, may be NULL; a bad request gets a zeroed block).  With
 * graph = 1 the first call with a given set of arguments captures the whole
 * sequence (scratch clears, binning kernels, decode kernel) into a CUDA graph
 * and later identical calls replay it.  Calls on one batch object share its
 * scratch: serialise them (one object per CUDA stream).  n = 0 is a no-op.
 * Errors: RLFC_E_INVALID_ARG (null pointer, level > L-1), RLFC_E_RANGE
 * (n > max_requests), RLFC_E_CUDA.
 */
RLFC_API int rlfc_batch_decode(rlfc_batch *b, const uint32_t *d_view, const uint32_t *d_loc, size_t n,
                               uint32_t level, uint8_t *d_out, uint8_t *d_status, void *cuda_stream);

/*
 * Time every candidate configuration (warps per CTA 4/8/16, locations per
 * pop 1/4, staging 0/1, and prefetching with one location per pop) on these
 * requests at level 0 with CUDA events,
 * keep the fastest (the graph flag is left as it was) and write it to
 * *chosen (may be NULL).  d_out and d_status receive the decoded requests.
 * Synchronises `cuda_stream`.  Errors: as rlfc_batch_decode.
 */
RLFC_API int rlfc_batch_autotune(rlfc_batch *b, const uint32_t *d_view, const uint32_t *d_loc, size_t n,
                                 uint8_t *d_out, uint8_t *d_status, void *cuda_stream,
                                 rlfc_batch_config *chosen);

/* Release a batch object.  Like rlfc_free_stream it first waits for the
 * device to finish its queued work. */
RLFC_API void rlfc_batch_free(rlfc_batch *b);

/*
 * Serving (the interactive use the paper targets, Sections 1 and 5: new
 * views of resident compressed light fields on demand; the paper has no
 * serving runtime of its own).  A server keeps loaded streams on the device
 * and runs one worker thread that batches view requests continuously:
 *  - rlfc_server_submit queues a request (light field, camera (u, v), focus
 *    disparity, output size, host destination) and returns at once;
 *  - the worker admits queued requests in arrival order while the device
 *    memory of their outputs fits the memory budget, groups the admitted ones
 *    by (light field, output size) into calls of rlfc_render_views of at most
 *    max_batch views, and issues each call on the least busy of n_streams
 *    CUDA streams that holds fewer than max_inflight calls, followed by the
 *    copy of every view to its host destination;
 *  - requests that arrive while earlier calls run are admitted as soon as
 *    memory frees, and their calls overlap the earlier ones on other streams;
 *  - a completed request (its copy to the host done) is reported by
 *    rlfc_server_poll with its submit, start and completion times (seconds on
 *    the clock of rlfc_server_now).
 * A view's pixels do not depend on which other requests shared its call, so
 * every result equals that of rendering the request alone.
 */
typedef struct rlfc_server rlfc_server;   /* opaque, library-owned */

typedef struct {
    uint32_t n_streams;       /* CUDA streams calls are spread over, 1..64 */
    uint32_t max_batch;       /* views per render call, 1..4096 */
    uint64_t memory_budget;   /* device bytes of outputs in flight (out_w*out_h*12 + 12 per float view, out_w*out_h*3 + 12 per 8-bit view) */
    uint32_t max_inflight;    /* calls queued on one stream at a time, 1..64: while every stream
                                 is full, arrivals wait and then share the next call */
    uint32_t pad;
} rlfc_server_config;

typedef struct {
    uint64_t ticket;          /* from rlfc_server_submit */
    int32_t status;           /* RLFC_OK or the render call's error code */
    uint32_t lf;              /* light-field id */
    uint32_t batch;           /* views in the call that served it */
    uint32_t pad;
    double t_submit, t_start, t_done;   /* rlfc_server_now() clock, seconds */
} rlfc_completion;

/* Start a server on the current CUDA device.  Errors: RLFC_E_INVALID_ARG,
 * RLFC_E_OOM, RLFC_E_CUDA. */
RLFC_API int rlfc_server_create(const rlfc_server_config *cfg, rlfc_server **out);

/* Make a loaded stream servable (it must be on the server's device and
 * outlive the server); *lf_id receives its id.  Errors: RLFC_E_INVALID_ARG. */
RLFC_API int rlfc_server_add(rlfc_server *srv, const rlfc_stream *s, uint32_t *lf_id);

/*
 * Queue one view request; host_out (out_h * out_w * 3 floats, ideally pinned)
 * receives the view and must stay valid until the request completes.
 * Thread-safe.  Errors: RLFC_E_INVALID_ARG (unknown id, null pointer, empty
 * size), RLFC_E_RANGE (one view larger than the memory budget or than
 * rlfc_render_views accepts).
 */
RLFC_API int rlfc_server_submit(rlfc_server *srv, uint32_t lf_id, float u, float v, float disp,
                                uint32_t out_w, uint32_t out_h, float *host_out, uint64_t *ticket);

/*
 * As rlfc_server_submit, with the view delivered as 8-bit RGB (out_h * out_w
 * * 3 bytes, the rounding of rlfc_render_views_u8): a quarter of the device
 * memory and of the copy to the host.  Requests of the two formats never
 * share a call.  Errors: as rlfc_server_submit.
 */
RLFC_API int rlfc_server_submit_u8(rlfc_server *srv, uint32_t lf_id, float u, float v, float disp,
                                   uint32_t out_w, uint32_t out_h, uint8_t *host_out, uint64_t *ticket);

/*
 * Move up to `cap` completed requests into out (oldest first) and set *n.
 * With wait != 0 the call first blocks until every submitted request has
 * completed.  Errors: RLFC_E_INVALID_ARG.
 */
RLFC_API int rlfc_server_poll(rlfc_server *srv, rlfc_completion *out, size_t cap, size_t *n, int wait);

/* Seconds on the server's monotonic clock. */
RLFC_API double rlfc_server_now(void);

/* Finish the queued requests, stop the worker and release the server. */
RLFC_API void rlfc_server_free(rlfc_server *srv);

/* Encoder parameters (Algorithm 1, Section 3.1-3.3). */
typedef struct {
    uint32_t U, V, W, H;  /* grid and view size */
    uint32_t B;           /* block side; the GPU encoder supports 4 */
    uint32_t L;           /* tree levels, 2..8 */
    uint32_t c[8];        /* cluster side used to build level l from l-1 (c[1..L-1]) */
    int32_t tau_p;        /* pixel threshold: |r| < tau_p is zeroed */
    int32_t tau_b;        /* block energy threshold: sum |r| < tau_b drops the block */
    uint32_t q;           /* global quantisation shift, 0..7 */
    /* block modes: 0 = the plain method (shift 0, the smallest range that holds
       the span); 1 = per block the (shift s, mode k) of least cost
       256 * payload bits + lam_q8 * SSE among the pairs whose range holds the
       span of qv = sign(r) floor((|r| + 2^(q+s-1)) / 2^(q+s)) and, for s > 0,
       whose error |r - qv 2^(q+s)| stays within tau_err (the header's shift
       field, reconstructed as qv 2^(q+s)); this mode space is the learned
       encoder aid's and has no counterpart in the paper */
    uint32_t mode_space;
    int32_t tau_err;
    uint32_t lam_q8;
} rlfc_enc_params;

/*
 * Algorithm 1 on the GPU: compress the views d_rgb (device, U*V*H*W*3 bytes,
 * views in index order, RGB rows) into a format-v1 stream.  Every rule is
 * integer arithmetic, so the output is byte-identical to any other encoder
 * that follows them:
 *  - views are padded to a multiple of B by repeating the last column / row
 *    and converted to YCoCg-R (Section 4);
 *  - level l's grid cuts level l-1's into k = ceil(G / c[l]) tiles per axis,
 *    tile a covering [floor(a G / k), floor((a + 1) G / k)) (Eq. 1);
 *  - a tile of mu x mv nodes is filtered with the binomial weights
 *    C(mu-1, i) C(mv-1, j): RKV = floor((sum w X + 2^(s-1)) / 2^s),
 *    s = mu + mv - 2 (Eq. 2);
 *  - top-down, r = child RKV - parent reconstruction (Eq. 3); |r| < tau_p is
 *    zeroed; a block whose sum |r| is below tau_b or zero is dropped; kept
 *    values are quantised to sign(r) floor((|r| + 2^(q-1)) / 2^q) (no rounding
 *    term when q = 0), a block quantising to all zeros is dropped, and the
 *    child's reconstruction is parent + qv 2^q (Section 3.2);
 *  - a stored block's header holds its minimum and the smallest mode whose
 *    range holds max - min + 1 values (the cheapest one).
 * On success *host_out holds *nbytes bytes allocated by the library
 * (free with rlfc_free_host); the call synchronises `cuda_stream`.
 * Errors: RLFC_E_INVALID_ARG, RLFC_E_UNSUPPORTED, RLFC_E_RANGE, RLFC_E_OOM,
 * RLFC_E_CUDA.
 */
RLFC_API int rlfc_encode(const rlfc_enc_params *p, const uint8_t *d_rgb, void *cuda_stream,
                void **host_out, size_t *nbytes);

/*
 * rlfc_encode with the learned encoder aid's hooks for the level-0 (view)
 * blocks, whose index is (view * 3 + channel) * nloc + location:
 *  - d_leaf_modes (device, may be NULL; mode_space 1 only): a given k | s << 5
 *    per block, used when it is a candidate (see rlfc_enc_params), otherwise
 *    and for 0xFF the search decides;
 *  - d_leaf_resid (device, may be NULL): receives each block's 16 residuals
 *    after the pixel threshold, int16;
 *  - d_leaf_label (device, may be NULL): receives the search's k | s << 5 for
 *    the blocks the energy test keeps, 0xFF for the others.
 * Errors: as rlfc_encode.
 */
RLFC_API int rlfc_encode_ex(const rlfc_enc_params *p, const uint8_t *d_rgb, const uint8_t *d_leaf_modes,
                            int16_t *d_leaf_resid, uint8_t *d_leaf_label, void *cuda_stream,
                            void **host_out, size_t *nbytes);

/*
 * The same encoder for callers that cannot allocate device memory while they
 * encode: code running under a custom or capped device allocator that must not
 * see foreign cudaMalloc calls, processes whose device memory is reserved up
 * front, or callers that must avoid the device-wide synchronisation of
 * cudaMalloc / cudaFree.  The paper has no counterpart; this is a deployment
 * variant of rlfc_encode with byte-identical output.
 *
 * It calls no cudaMalloc, cudaFree or other device-allocating routine.  Its
 * device scratch is one array of 32 MiB compiled into the library.  Under
 * lazy module loading (the CUDA default) a device holds it from the first
 * call on that device until the process exits; with
 * CUDA_MODULE_LOADING=EAGER every context that loads the library holds it
 * from its creation.
 * Light fields whose encoder scratch exceeds 32 MiB (roughly up to 9 x 9
 * views of 128 x 128, depending on the tree) are rejected with RLFC_E_RANGE
 * before any work is enqueued; use rlfc_encode for those.
 *
 * The caller passes the input views d_rgb (as for rlfc_encode) and a host
 * buffer host_out of `capacity` bytes.  On success *nbytes holds the stream
 * size and host_out the stream; if the buffer is too small the call returns
 * RLFC_E_RANGE with *nbytes set to the size needed.
 *
 * Every call looks up the array's device address (cudaGetSymbolAddress) in
 * the current context, so a device reset between calls is harmless; under
 * lazy loading the first call on a device also loads the array's module.
 * The encoder carves its buffers from the first bytes of the array, at most
 * the bound that the size check computed, and fails with RLFC_E_CUDA rather
 * than use more.  Every call shares the one array and leaves its
 * contents behind (the words that must start at zero are cleared on every
 * call), so calls that overlap on the GPU, from several host threads or
 * streams, race and must be serialised by the caller.  The call synchronises
 * `cuda_stream`.  Errors: RLFC_E_INVALID_ARG, RLFC_E_UNSUPPORTED, RLFC_E_RANGE,
 * RLFC_E_CUDA.
 */
RLFC_API int rlfc_encode_no_alloc(const rlfc_enc_params *p, const uint8_t *d_rgb, void *cuda_stream,
                                  void *host_out, size_t capacity, size_t *nbytes);

/*
 * Kernel tracing (a profiling aid; the paper has no counterpart).  While
 * tracing is on, every kernel the library launches outside stream capture is
 * bracketed by two CUDA events on its launching stream, and the durations are
 * summed per kernel name.  rlfc_trace_read waits for the traced work, then
 * writes up to `cap` entries (one per kernel name seen since the last reset)
 * and sets *n to the number of names; with reset != 0 the totals restart
 * from zero.  Tracing adds two event records per launch; leave it off when
 * timing whole calls.  Errors: RLFC_E_INVALID_ARG, RLFC_E_CUDA.
 */
typedef struct {
    char kernel[56];     /* kernel name, NUL-terminated */
    uint64_t launches;   /* traced launches */
    double total_ms;     /* summed event-to-event durations */
} rlfc_trace_entry;

RLFC_API int rlfc_trace_enable(int on);
RLFC_API int rlfc_trace_read(rlfc_trace_entry *out, size_t cap, size_t *n, int reset);

/*
 * Learned encoder aid (no counterpart in the paper; it sits beside the encoder
 * and never changes how a stream decodes).  A small network predicts each
 * level-0 block's (shift, mode) from 48 statistics of its residuals; the
 * exhaustive search stays the arbiter and the fallback (rlfc_encode_ex takes a
 * predicted mode only when it is a candidate).  All pointers are device
 * pointers; every call is asynchronous on `cuda_stream`.
 *
 * Network: 48 -> 64 (ReLU) -> 64 (ReLU) -> 112 logits, class s * 28 + k.
 * Parameters (RLFC_MLP_PARAMS, flat, in this order): W1 [64][48], b1 [64],
 * W2 [64][64], b2 [64], W3 [112][64], b3 [112] (rows are output units), stored
 * as BF16 (uint16 bit patterns); products and sums are FP32.
 * Labels are header bytes k | s << 5.
 */
#define RLFC_KS_FEATURES 48
#define RLFC_KS_CLASSES 112
#define RLFC_MLP_PARAMS 14576

/* The search of rlfc_enc_params for n blocks of 16 int16 residuals:
 * d_label[i] = k | s << 5, or 0xFF when no pair is a candidate.
 * Errors: RLFC_E_INVALID_ARG, RLFC_E_RANGE (n >= 2^31), RLFC_E_CUDA. */
RLFC_API int rlfc_ks_search(const int16_t *d_resid, size_t n, uint32_t q, int32_t tau_err, uint32_t lam_q8,
                            uint8_t *d_label, void *cuda_stream);

/* Positions of the entries of d_label[0..n) that are not 0xFF, ascending,
 * into d_index; their number into *d_count (device).  Errors: as above. */
RLFC_API int rlfc_ks_compact(const uint8_t *d_label, size_t n, uint32_t *d_index, uint32_t *d_count,
                             void *cuda_stream);

/* The 48 statistics (BF16) of blocks d_resid[d_index[i]] (or [i] when
 * d_index is NULL) into d_x [n][48]: the values sorted ascending / 32, the
 * values in raster order / 32, mean, standard deviation, min, max / 32,
 * span / 64, max |r| / 32, sum |r| / 256, the counts of non-zero, odd,
 * 2 (mod 4), 4 (mod 8), |r| <= 1, 2, 4, 8 values / 16, log2(span + 1) / 10.
 * d_label_out (may be NULL) receives d_label[d_index[i]].  Errors: as above. */
RLFC_API int rlfc_ks_features(const int16_t *d_resid, const uint8_t *d_label, const uint32_t *d_index, size_t n,
                              uint16_t *d_x, uint8_t *d_label_out, void *cuda_stream);

/* Training step, forward and backward: for the samples d_order[0..n) (or
 * 0..n) of (d_x, d_label), add the summed softmax cross-entropy to *d_loss
 * and its summed gradient to d_grad [RLFC_MLP_PARAMS] (FP32; sums over CTAs
 * use atomics, so the last bits vary between runs).  Labels whose mode is not
 * below 28 are skipped.  Errors: as above. */
RLFC_API int rlfc_mlp_loss_grad(const uint16_t *d_w, const uint16_t *d_x, const uint8_t *d_label,
                                const uint32_t *d_order, size_t n, float *d_grad, float *d_loss, void *cuda_stream);

/* Adam update of the FP32 master parameters from grad * grad_scale (step =
 * 1, 2, ... for the bias corrections), refreshing the BF16 copy d_w and
 * clearing d_grad.  Errors: RLFC_E_INVALID_ARG, RLFC_E_CUDA. */
RLFC_API int rlfc_mlp_adam(float *d_master, uint16_t *d_w, float *d_grad, float *d_m, float *d_v, float lr,
                           float beta1, float beta2, float eps, float grad_scale, uint32_t step, void *cuda_stream);

/* Inference: the predicted label (first largest logit) of each sample i goes
 * to d_label[d_index[i]] (or [i]).  Errors: as rlfc_ks_search. */
RLFC_API int rlfc_mlp_predict(const uint16_t *d_w, const uint16_t *d_x, size_t n, const uint32_t *d_index,
                              uint8_t *d_label, void *cuda_stream);

/*
 * Debug builds: the flags the device bounds checks raised for stream s.
 *
 * A library built with RLFC_DEBUG (the build script's debug option) checks,
 * in the full decode, the per-request decode, the binned decode and the
 * renderer's on-demand decode, every stored block before it is decoded: its mode index is one of the 28 BISE
 * modes, its 18-bit header lies in its record's header area, and its payload
 * lies inside its record (Algorithm 2's record layout, Section 3.4); the
 * full decode also checks every output view index.  A failed check sets a
 * bit in a flag word the stream owns and the block is treated as absent (the
 * output view is skipped): nothing is read or written out of range and no
 * kernel traps.  Bits: 1 mode, 2 header, 4 payload, 8 output index.  The
 * loader validates every record, so a stream it accepted raises no flag;
 * the checks guard the decoders' own index arithmetic, in place of a memory
 * checker.
 *
 * Writes the flags to *flags (host memory) after the device has finished
 * the work queued so far (the call synchronises the device), and clears them
 * when reset is nonzero.  The paper has no counterpart.  Errors:
 * RLFC_E_INVALID_ARG (null s or flags), RLFC_E_UNSUPPORTED (a release build,
 * *flags = 0), RLFC_E_CUDA.
 */
RLFC_API int rlfc_debug_flags(const rlfc_stream *s, uint32_t *flags, int reset);

/* Free a host buffer returned by the library. */
RLFC_API void rlfc_free_host(void *p);

/* Static description of a status code. */
RLFC_API const char *rlfc_strerror(int code);

/* Detail of the most recent failure on the calling thread ("" if none). */
RLFC_API const char *rlfc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* RLFC_H */

// The learned encoder aid: per-block (shift, mode) search, the 48 block
// statistics, and a 48 -> 64 -> 64 -> 112 perceptron with its training
// (forward, softmax cross-entropy, backward, Adam) and inference kernels.
//
// Numerics: parameters and inputs are stored in BF16; sums and activations
// are FP32.  The network is small (14 576 parameters, layers 48 to 112 wide),
// so the kernels keep the transposed weights, the gradient accumulators and
// one tile of 32 samples' activations in shared memory; the products run on
// the tensor pipe (BF16 MMA with FP32 accumulation, FP32 operands split into
// two BF16 terms; see the tile helpers below).
//
// Parameter order (flat): W1 [64][48], b1 [64], W2 [64][64], b2 [64],
// W3 [112][64], b3 [112]; rows are output units.  Class c = s * 28 + k.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "rlfc_device.cuh"
#include "rlfc_internal.h"

namespace rlfc {
namespace {

__constant__ uint32_t c_rangeN[kNumModes] = {1,  2,  3,  4,   5,   6,   8,   10,  12,  16,  20,  24,  32,  40,
                                             48, 64, 80, 96, 128, 160, 192, 256, 320, 384, 512, 640, 768, 1024};
__constant__ uint32_t c_modes[kNumModes] = RLFC_MODE_TABLE_INIT;

#include "ks_device.cuh"

constexpr int NI = 48, NH = 64, NO = 112;
constexpr int kP = NH * NI + NH + NH * NH + NH + NO * NH + NO;   // 14576
constexpr int oW1 = 0, oB1 = NH * NI, oW2 = oB1 + NH, oB2 = oW2 + NH * NH, oW3 = oB2 + NH, oB3 = oW3 + NO * NH;
constexpr int kTile = 32;
constexpr int kThreads = 256;
constexpr unsigned kFull = 0xFFFFFFFFu;

__device__ __forceinline__ float bf(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }
__device__ __forceinline__ uint16_t to_bf(float f) { return __bfloat16_as_ushort(__float2bfloat16_rn(f)); }

__global__ void ks_search_kernel(const int16_t *resid, uint32_t n, uint32_t q, int32_t tau_err, uint32_t lam_q8,
                                 uint8_t *label)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    int r[kVals];
#pragma unroll
    for (int k = 0; k < kVals; k++)
        r[k] = resid[(size_t)i * kVals + k];
    uint32_t k = 0, s = 0;
    label[i] = ks_search(r, q, tau_err, lam_q8, k, s) ? (uint8_t)(k | s << 5) : (uint8_t)0xFF;
}

// Compaction of the entries != 0xFF, in ascending order: per-chunk counts,
// then each chunk writes at the sum of the counts before it.
constexpr uint32_t kChunk = 4096;

__global__ void __launch_bounds__(1024) compact_count_kernel(const uint8_t *label, uint32_t n, uint32_t *part)
{
    __shared__ uint32_t s_w[32];
    uint32_t c = 0;
    for (uint32_t k = 0; k < kChunk / 1024; k++) {
        const uint32_t i = blockIdx.x * kChunk + k * 1024 + threadIdx.x;
        c += i < n && label[i] != 0xFF;
    }
    c = __reduce_add_sync(kFull, c);
    if ((threadIdx.x & 31) == 0)
        s_w[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x < 32) {
        const uint32_t t = __reduce_add_sync(kFull, s_w[threadIdx.x]);
        if (threadIdx.x == 0)
            part[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(1024) compact_write_kernel(const uint8_t *label, uint32_t n, const uint32_t *part,
                                                             uint32_t *index, uint32_t *count)
{
    __shared__ uint32_t s_w[32];
    __shared__ uint32_t s_base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        uint32_t b = 0;
        for (uint32_t c = 0; c < blockIdx.x; c++)
            b += part[c];
        s_base = b;
        if (blockIdx.x == gridDim.x - 1)
            *count = b + part[blockIdx.x];
    }
    __syncthreads();
    uint32_t base = s_base;
    for (uint32_t k = 0; k < kChunk / 1024; k++) {
        const uint32_t i = blockIdx.x * kChunk + k * 1024 + threadIdx.x;
        const bool keep = i < n && label[i] != 0xFF;
        const uint32_t bal = __ballot_sync(kFull, keep);
        if (lane == 0)
            s_w[warp] = __popc(bal);
        __syncthreads();
        uint32_t before = 0, total = 0;
        for (int w = 0; w < 32; w++) {
            before += w < warp ? s_w[w] : 0u;
            total += s_w[w];
        }
        if (keep)
            index[base + before + __popc(bal & ((1u << lane) - 1u))] = i;
        base += total;
        __syncthreads();
    }
}

__device__ __forceinline__ void sort16(int v[16])
{
    // insertion sort in registers
#pragma unroll
    for (int i = 1; i < 16; i++) {
#pragma unroll
        for (int j = i; j > 0; j--) {
            const int a = v[j - 1], b = v[j];
            v[j - 1] = min(a, b);
            v[j] = max(a, b);
        }
    }
}

// The 48 statistics of each block (order and scaling as in the aid's
// definition): sorted values / 32, raw values / 32, mean, standard
// deviation, min, max / 32, span / 64, max |r| / 32, sum |r| / 256, and the
// counts of non-zero, odd, 2 (mod 4), 4 (mod 8), |r| <= 1, 2, 4, 8 values / 16,
// log2(span + 1) / 10.
__global__ void ks_features_kernel(const int16_t *resid, const uint8_t *label_in, const uint32_t *index, uint32_t n,
                                   uint16_t *x, uint8_t *label_out)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    const size_t src = index ? index[i] : i;
    int r[16], sorted[16];
    int sum = 0, sum2 = 0, l1 = 0, mn = 0, mx = 0, amax = 0, nz = 0, odd = 0, m4 = 0, m8 = 0;
    int le1 = 0, le2 = 0, le4 = 0, le8 = 0;
#pragma unroll
    for (int k = 0; k < 16; k++) {
        const int v = resid[src * 16 + k];
        r[k] = sorted[k] = v;
        const int a = abs(v);
        sum += v;
        sum2 += v * v;
        l1 += a;
        mn = k == 0 ? v : min(mn, v);
        mx = k == 0 ? v : max(mx, v);
        amax = max(amax, a);
        nz += v != 0;
        odd += a & 1;
        m4 += (a & 3) == 2;
        m8 += (a & 7) == 4;
        le1 += a <= 1;
        le2 += a <= 2;
        le4 += a <= 4;
        le8 += a <= 8;
    }
    sort16(sorted);
    uint16_t *o = x + (size_t)i * NI;
#pragma unroll
    for (int k = 0; k < 16; k++) {
        o[k] = to_bf((float)sorted[k] / 32.0f);
        o[16 + k] = to_bf((float)r[k] / 32.0f);
    }
    const float mean = (float)sum / 16.0f;
    const float var = fmaxf((float)sum2 / 16.0f - mean * mean, 0.0f);
    o[32] = to_bf(mean / 32.0f);
    o[33] = to_bf(sqrtf(var) / 32.0f);
    o[34] = to_bf((float)mn / 32.0f);
    o[35] = to_bf((float)mx / 32.0f);
    o[36] = to_bf((float)(mx - mn) / 64.0f);
    o[37] = to_bf((float)amax / 32.0f);
    o[38] = to_bf((float)l1 / 256.0f);
    o[39] = to_bf((float)nz / 16.0f);
    o[40] = to_bf((float)odd / 16.0f);
    o[41] = to_bf((float)m4 / 16.0f);
    o[42] = to_bf((float)m8 / 16.0f);
    o[43] = to_bf((float)le1 / 16.0f);
    o[44] = to_bf((float)le2 / 16.0f);
    o[45] = to_bf((float)le4 / 16.0f);
    o[46] = to_bf((float)le8 / 16.0f);
    o[47] = to_bf(log2f((float)(mx - mn) + 1.0f) / 10.0f);
    if (label_out)
        label_out[i] = label_in ? label_in[src] : (uint8_t)0xFF;
}

// ---- BF16 tensor-core tiles -------------------------------------------------
//
// Every product of the network runs on the tensor pipe: mma.sync m16n8k16
// with BF16 operands and FP32 accumulation.  The weights and the inputs are
// BF16 values already (one term); an FP32 activation or delta is split into
// a BF16 high part and a BF16 residual, hi + lo, which carries 16 bits of its
// mantissa, so that a product with a weight is hi * w + lo * w (two MMAs) and
// a product of two FP32 operands hi * hi' + hi * lo' + lo * hi' (three).  The
// results then differ from FP32 arithmetic by a few units of 2^-16.
//
// Fragments (per lane, g = lane / 4, t = lane % 4): A (16 x 16, row-major)
// holds A[g][k..k+1], A[g+8][k..k+1], A[g][k+8..k+9], A[g+8][k+8..k+9] with
// k = 2t; B (16 x 8) holds B[2t..2t+1][g], B[2t+8..2t+9][g]; C (16 x 8)
// holds C[g][2t..2t+1], C[g+8][2t..2t+1].  Pairs are packed low element
// first.

__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], const uint32_t b[2])
{
    asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Two floats to a BF16 pair (x0 in the low half), rounded to nearest.
__device__ __forceinline__ uint32_t pack_bf16(float x0, float x1)
{
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(x1), "f"(x0));
    return r;
}

// hi = bf16(x), lo = bf16(x - hi), for a pair.
__device__ __forceinline__ void split2(float x0, float x1, uint32_t &hi, uint32_t &lo)
{
    hi = pack_bf16(x0, x1);
    lo = pack_bf16(x0 - __uint_as_float(hi << 16), x1 - __uint_as_float(hi & 0xFFFF0000u));
}

// Leading dimensions (floats) of the FP32 activation tiles: 4 mod 16 keeps
// the column-wise fragment loads on distinct banks.
constexpr int LX = NI + 4, LH = NH + 4, LZ = NO + 4;
// Row strides (BF16 elements) of the weight copies: the row-wise fragment
// loads fall on distinct banks.
constexpr int LW1 = NI + 8, LW2 = NH + 8, LW3 = NH + 8, LW2T = NH + 8, LW3T = NO + 8;

// A fragment of a row-major FP32 tile M[m][k] (rows m0.., columns k0..).
template <bool kExact>
__device__ __forceinline__ void frag_a_rows(const float *M, int ld, int m0, int k0, uint32_t hi[4], uint32_t lo[4])
{
    const int g = (threadIdx.x & 31) >> 2, t = threadIdx.x & 3;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const float2 v = *reinterpret_cast<const float2 *>(M + (m0 + g + 8 * (q & 1)) * ld + k0 + 2 * t + 8 * (q >> 1));
        if (kExact)
            hi[q] = pack_bf16(v.x, v.y);
        else
            split2(v.x, v.y, hi[q], lo[q]);
    }
}

// A fragment of the transpose of an FP32 tile: A[m][k] = M[k][m].
__device__ __forceinline__ void frag_a_cols(const float *M, int ld, int m0, int k0, uint32_t hi[4], uint32_t lo[4])
{
    const int g = (threadIdx.x & 31) >> 2, t = threadIdx.x & 3;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const int m = m0 + g + 8 * (q & 1), k = k0 + 2 * t + 8 * (q >> 1);
        split2(M[k * ld + m], M[(k + 1) * ld + m], hi[q], lo[q]);
    }
}

// B fragment of BF16 weights stored n-major, B[k][n] = Wb[n][k] (row stride ldw).
__device__ __forceinline__ void frag_b_w(const uint16_t *Wb, int ldw, int n0, int k0, uint32_t b[2])
{
    const int g = (threadIdx.x & 31) >> 2, t = threadIdx.x & 3;
    const uint32_t *row = reinterpret_cast<const uint32_t *>(Wb + (n0 + g) * ldw + k0);
    b[0] = row[t];
    b[1] = row[4 + t];
}

// B fragment of a row-major FP32 tile, B[k][n] = M[k][n].
template <bool kExact>
__device__ __forceinline__ void frag_b_rows(const float *M, int ld, int n0, int k0, uint32_t hi[2], uint32_t lo[2])
{
    const int g = (threadIdx.x & 31) >> 2, t = threadIdx.x & 3;
#pragma unroll
    for (int q = 0; q < 2; q++) {
        const int k = k0 + 2 * t + 8 * q;
        const float x0 = M[k * ld + n0 + g], x1 = M[(k + 1) * ld + n0 + g];
        if (kExact)
            hi[q] = pack_bf16(x0, x1);
        else
            split2(x0, x1, hi[q], lo[q]);
    }
}

// C tile (16 x 8) at (m0, n0) of act(b + X W^T): X an FP32 activation tile
// [m][K] (row stride ldx; BF16 values exactly when kXExact), W BF16 weights
// [N][K], stored into Y (row stride ldy).
template <int K, bool kXExact, bool kRelu>
__device__ __forceinline__ void dense_tile(const float *X, int ldx, const uint16_t *Wb, int ldw, const float *b,
                                           float *Y, int ldy, int m0, int n0)
{
    float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int k0 = 0; k0 < K; k0 += 16) {
        uint32_t ah[4], al[4], bw[2];
        frag_a_rows<kXExact>(X, ldx, m0, k0, ah, al);
        frag_b_w(Wb, ldw, n0, k0, bw);
        mma_bf16(c, ah, bw);
        if (!kXExact)
            mma_bf16(c, al, bw);
    }
    const int g = (threadIdx.x & 31) >> 2, t = threadIdx.x & 3, n = n0 + 2 * t;
    const float b0 = b[n], b1 = b[n + 1];
    float y[4] = {c[0] + b0, c[1] + b1, c[2] + b0, c[3] + b1};
    if (kRelu)
        for (int q = 0; q < 4; q++)
            y[q] = fmaxf(y[q], 0.0f);
    *reinterpret_cast<float2 *>(Y + (m0 + g) * ldy + n) = make_float2(y[0], y[1]);
    *reinterpret_cast<float2 *>(Y + (m0 + g + 8) * ldy + n) = make_float2(y[2], y[3]);
}

// The network's weights in shared memory: BF16 copies for the fragments
// (W1, W2, W3 row-major as stored, W2 and W3 transposed for the backward
// pass) and FP32 biases.
struct NetW {
    uint16_t *w1, *w2, *w3, *w2t, *w3t;
    float *b1, *b2, *b3;
};

constexpr int kWBytes = 2 * (NH * LW1 + NH * LW2 + NO * LW3 + NH * LW2T + NH * LW3T) + 4 * (NH + NH + NO);

__device__ __forceinline__ NetW carve_w(unsigned char *base, bool transposed)
{
    NetW m;
    m.w1 = reinterpret_cast<uint16_t *>(base);
    m.w2 = m.w1 + NH * LW1;
    m.w3 = m.w2 + NH * LW2;
    m.w2t = m.w3 + NO * LW3;
    m.w3t = m.w2t + (transposed ? NH * LW2T : 0);
    float *f = reinterpret_cast<float *>(m.w3t + (transposed ? NH * LW3T : 0));
    m.b1 = f;
    m.b2 = f + NH;
    m.b3 = f + 2 * NH;
    return m;
}

__device__ void load_weights(const uint16_t *w, const NetW &m, bool transposed)
{
    for (int i = threadIdx.x; i < NH * NI; i += blockDim.x)
        m.w1[(i / NI) * LW1 + i % NI] = w[oW1 + i];
    for (int i = threadIdx.x; i < NH * NH; i += blockDim.x) {
        const int j = i / NH, k = i % NH;
        m.w2[j * LW2 + k] = w[oW2 + i];
        if (transposed)
            m.w2t[k * LW2T + j] = w[oW2 + i];
    }
    for (int i = threadIdx.x; i < NO * NH; i += blockDim.x) {
        const int j = i / NH, k = i % NH;
        m.w3[j * LW3 + k] = w[oW3 + i];
        if (transposed)
            m.w3t[k * LW3T + j] = w[oW3 + i];
    }
    for (int i = threadIdx.x; i < NH; i += blockDim.x) {
        m.b1[i] = bf(w[oB1 + i]);
        m.b2[i] = bf(w[oB2 + i]);
    }
    for (int i = threadIdx.x; i < NO; i += blockDim.x)
        m.b3[i] = bf(w[oB3 + i]);
}

// Tile of samples [t0, t0 + kTile) in `order` (or in index order): inputs
// (FP32 copies of the BF16 values) and classes (-1 for missing or invalid
// ones).
__device__ __forceinline__ void load_tile(const uint16_t *x, const uint8_t *label, const uint32_t *order,
                                          uint32_t n, uint32_t t0, float *X, int *s_cls)
{
    for (int i = threadIdx.x; i < kTile * NI; i += blockDim.x) {
        const uint32_t s = i / NI, f = i % NI, gs = t0 + s;
        float v = 0.0f;
        if (gs < n)
            v = bf(x[(size_t)(order ? order[gs] : gs) * NI + f]);
        X[s * LX + f] = v;
    }
    if (s_cls && threadIdx.x < kTile) {
        const uint32_t gs = t0 + threadIdx.x;
        int c = -1;
        if (gs < n) {
            const uint32_t lab = label[order ? order[gs] : gs];
            if ((lab & 31u) < (uint32_t)kNumModes)
                c = (int)((lab >> 5) * kNumModes + (lab & 31u));
        }
        s_cls[threadIdx.x] = c;
    }
}

// Gradient tile (16 x 8) at (m0, n0) of A^T B over the tile's samples,
// A = D [s][m] (deltas, row stride ldd) and B = H [s][n] (activations or
// inputs, row stride ldh), added to G[m][n] (row stride ldg).
template <bool kHExact>
__device__ __forceinline__ void grad_tile(const float *D, int ldd, const float *H, int ldh, float *G, int ldg, int m0,
                                          int n0)
{
    float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int k0 = 0; k0 < kTile; k0 += 16) {
        uint32_t ah[4], al[4], bh[2], bl[2];
        frag_a_cols(D, ldd, m0, k0, ah, al);
        frag_b_rows<kHExact>(H, ldh, n0, k0, bh, bl);
        mma_bf16(c, ah, bh);
        mma_bf16(c, al, bh);
        if (!kHExact)
            mma_bf16(c, ah, bl);
    }
    const int g = (threadIdx.x & 31) >> 2, t = threadIdx.x & 3;
    float *r0 = G + (m0 + g) * ldg + n0 + 2 * t, *r1 = r0 + 8 * ldg;
    r0[0] += c[0];
    r0[1] += c[1];
    r1[0] += c[2];
    r1[1] += c[3];
}

// Delta tile (16 x 8) at (m0, n0) of (Dn Wn) * relu'(H): Dn the next layer's
// deltas [s][K] (row stride ldd), Wn^T as BF16 weights [N][K], H the layer's
// activations [s][N].
template <int K>
__device__ __forceinline__ void delta_tile(const float *Dn, int ldd, const uint16_t *Wt, int ldw, const float *H,
                                           int ldh, float *D, int ld, int m0, int n0)
{
    float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int k0 = 0; k0 < K; k0 += 16) {
        uint32_t ah[4], al[4], bw[2];
        frag_a_rows<false>(Dn, ldd, m0, k0, ah, al);
        frag_b_w(Wt, ldw, n0, k0, bw);
        mma_bf16(c, ah, bw);
        mma_bf16(c, al, bw);
    }
    const int g = (threadIdx.x & 31) >> 2, t = threadIdx.x & 3, n = n0 + 2 * t;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const int m = m0 + g + 8 * (q >> 1), nn = n + (q & 1);
        D[m * ld + nn] = H[m * ldh + nn] > 0.0f ? c[q] : 0.0f;
    }
}

constexpr int kTileFloats = kTile * (LX + LH + LH + LZ + LH + LH);

__global__ void __launch_bounds__(kThreads) mlp_loss_grad_kernel(const uint16_t *w, const uint16_t *x,
                                                                  const uint8_t *label, const uint32_t *order,
                                                                  uint32_t n, float *grad, float *loss)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_cls[kTile];
    __shared__ float s_loss;
    const NetW m = carve_w(smem, true);
    float *X = reinterpret_cast<float *>(smem + kWBytes);
    float *H1 = X + kTile * LX, *H2 = H1 + kTile * LH, *Z = H2 + kTile * LH, *D2 = Z + kTile * LZ, *D1 = D2 + kTile * LH;
    float *g = D1 + kTile * LH;   // [kP] gradient accumulators, flat parameter order
    load_weights(w, m, true);
    for (int i = threadIdx.x; i < kP; i += blockDim.x)
        g[i] = 0.0f;
    if (threadIdx.x == 0)
        s_loss = 0.0f;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int kWarps = kThreads / 32, kM = kTile / 16;
    const uint32_t ntiles = (n + kTile - 1) / kTile;
    for (uint32_t tt = blockIdx.x; tt < ntiles; tt += gridDim.x) {
        load_tile(x, label, order, n, tt * kTile, X, s_cls);
        __syncthreads();
        // forward: 16 x 8 output tiles spread over the warps
        for (int q = warp; q < kM * (NH / 8); q += kWarps)
            dense_tile<NI, true, true>(X, LX, m.w1, LW1, m.b1, H1, LH, 16 * (q % kM), 8 * (q / kM));
        __syncthreads();
        for (int q = warp; q < kM * (NH / 8); q += kWarps)
            dense_tile<NH, false, true>(H1, LH, m.w2, LW2, m.b2, H2, LH, 16 * (q % kM), 8 * (q / kM));
        __syncthreads();
        for (int q = warp; q < kM * (NO / 8); q += kWarps)
            dense_tile<NH, false, false>(H2, LH, m.w3, LW3, m.b3, Z, LZ, 16 * (q % kM), 8 * (q / kM));
        __syncthreads();
        // softmax cross-entropy; Z becomes d loss / d z
        for (int s = warp; s < kTile; s += kWarps) {
            float *z = Z + s * LZ;
            const int y = s_cls[s];
            float zmax = -INFINITY;
            for (int j = lane; j < NO; j += 32)
                zmax = fmaxf(zmax, z[j]);
#pragma unroll
            for (int d = 16; d > 0; d >>= 1)
                zmax = fmaxf(zmax, __shfl_xor_sync(kFull, zmax, d));
            float den = 0.0f;
            for (int j = lane; j < NO; j += 32)
                den += expf(z[j] - zmax);
#pragma unroll
            for (int d = 16; d > 0; d >>= 1)
                den += __shfl_xor_sync(kFull, den, d);
            if (lane == 0 && y >= 0)
                atomicAdd(&s_loss, logf(den) + zmax - z[y]);
            __syncwarp();
            for (int j = lane; j < NO; j += 32)
                z[j] = y >= 0 ? expf(z[j] - zmax) / den - (j == y ? 1.0f : 0.0f) : 0.0f;
        }
        __syncthreads();
        // layer 3: gW3 += dz^T h2 (112 x 64), gb3; d2 = (dz W3) relu'(h2)
        for (int q = warp; q < (NO / 16) * (NH / 8); q += kWarps)
            grad_tile<false>(Z, LZ, H2, LH, g + oW3, NH, 16 * (q % (NO / 16)), 8 * (q / (NO / 16)));
        for (int q = warp; q < kM * (NH / 8); q += kWarps)
            delta_tile<NO>(Z, LZ, m.w3t, LW3T, H2, LH, D2, LH, 16 * (q % kM), 8 * (q / kM));
        for (int j = threadIdx.x; j < NO; j += kThreads) {
            float a = 0.0f;
            for (int s = 0; s < kTile; s++)
                a += Z[s * LZ + j];
            g[oB3 + j] += a;
        }
        __syncthreads();
        // layer 2: gW2 += d2^T h1 (64 x 64), gb2; d1 = (d2 W2) relu'(h1)
        for (int q = warp; q < (NH / 16) * (NH / 8); q += kWarps)
            grad_tile<false>(D2, LH, H1, LH, g + oW2, NH, 16 * (q % (NH / 16)), 8 * (q / (NH / 16)));
        for (int q = warp; q < kM * (NH / 8); q += kWarps)
            delta_tile<NH>(D2, LH, m.w2t, LW2T, H1, LH, D1, LH, 16 * (q % kM), 8 * (q / kM));
        for (int j = threadIdx.x; j < NH; j += kThreads) {
            float a = 0.0f;
            for (int s = 0; s < kTile; s++)
                a += D2[s * LH + j];
            g[oB2 + j] += a;
        }
        __syncthreads();
        // layer 1: gW1 += d1^T x (64 x 48), gb1
        for (int q = warp; q < (NH / 16) * (NI / 8); q += kWarps)
            grad_tile<true>(D1, LH, X, LX, g + oW1, NI, 16 * (q % (NH / 16)), 8 * (q / (NH / 16)));
        for (int j = threadIdx.x; j < NH; j += kThreads) {
            float a = 0.0f;
            for (int s = 0; s < kTile; s++)
                a += D1[s * LH + j];
            g[oB1 + j] += a;
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < kP; i += blockDim.x)
        atomicAdd(&grad[i], g[i]);
    if (threadIdx.x == 0)
        atomicAdd(loss, s_loss);
}

// Inference: each warp takes 16 samples at a time through the three layers
// on its own activation tiles (no barrier after the weights are loaded),
// then takes the first maximum of each sample's logits.
constexpr int kPredWarpFloats = 16 * (LX + LH + LH + LZ);

__global__ void __launch_bounds__(kThreads) mlp_predict_kernel(const uint16_t *w, const uint16_t *x, uint32_t n,
                                                                const uint32_t *index, uint8_t *label)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const NetW m = carve_w(smem, false);
    load_weights(w, m, false);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float *X = reinterpret_cast<float *>(smem + kWBytes) + warp * kPredWarpFloats;
    float *H1 = X + 16 * LX, *H2 = H1 + 16 * LH, *Z = H2 + 16 * LH;
    const uint32_t ngroups = (n + 15) / 16;
    for (uint32_t grp = blockIdx.x * (kThreads / 32) + warp; grp < ngroups; grp += gridDim.x * (kThreads / 32)) {
        const uint32_t s0 = 16 * grp;
        for (int i = lane; i < 16 * NI; i += 32) {
            const int q = i / NI, f = i - q * NI;
            X[q * LX + f] = s0 + q < n ? bf(x[(size_t)(s0 + q) * NI + f]) : 0.0f;
        }
        __syncwarp();
#pragma unroll 1
        for (int nt = 0; nt < NH / 8; nt++)
            dense_tile<NI, true, true>(X, LX, m.w1, LW1, m.b1, H1, LH, 0, 8 * nt);
        __syncwarp();
#pragma unroll 1
        for (int nt = 0; nt < NH / 8; nt++)
            dense_tile<NH, false, true>(H1, LH, m.w2, LW2, m.b2, H2, LH, 0, 8 * nt);
        __syncwarp();
#pragma unroll 1
        for (int nt = 0; nt < NO / 8; nt++)
            dense_tile<NH, false, false>(H2, LH, m.w3, LW3, m.b3, Z, LZ, 0, 8 * nt);
        __syncwarp();
        // first maximum of each sample's logits: lanes 2q, 2q + 1 take sample q
        {
            const int q = lane >> 1, half = lane & 1;
            float best = -INFINITY;
            int arg = 0;
            for (int j = half; j < NO; j += 2) {
                const float v = Z[q * LZ + j];
                if (v > best) {
                    best = v;
                    arg = j;
                }
            }
            const float ob = __shfl_xor_sync(kFull, best, 1);
            const int oa = __shfl_xor_sync(kFull, arg, 1);
            if (ob > best || (ob == best && oa < arg)) {
                best = ob;
                arg = oa;
            }
            const uint32_t gi = s0 + q;
            if (half == 0 && gi < n)
                label[index ? index[gi] : gi] = (uint8_t)((arg % kNumModes) | (arg / kNumModes) << 5);
        }
        __syncwarp();   // the next group overwrites this warp's tiles
    }
}

__global__ void mlp_adam_kernel(float *master, uint16_t *w, float *grad, float *m1, float *m2, float lr, float b1,
                                float b2, float eps, float scale, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kP)
        return;
    const float gv = grad[i] * scale;
    const float a = b1 * m1[i] + (1.0f - b1) * gv;
    const float v = b2 * m2[i] + (1.0f - b2) * gv * gv;
    m1[i] = a;
    m2[i] = v;
    const float p = master[i] - lr * (a / c1) / (sqrtf(v / c2) + eps);
    master[i] = p;
    w[i] = to_bf(p);
    grad[i] = 0.0f;
}

int net_grid(uint32_t n, int dev_sms)
{
    const uint32_t tiles = (n + kTile - 1) / kTile;
    return (int)std::max<uint32_t>(1, std::min<uint32_t>(tiles, (uint32_t)dev_sms));
}

int sm_count()
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return std::max(v, 1);
}

}  // namespace
}  // namespace rlfc

extern "C" {

RLFC_API int rlfc_ks_search(const int16_t *d_resid, size_t n, uint32_t q, int32_t tau_err, uint32_t lam_q8,
                            uint8_t *d_label, void *cuda_stream)
{
    using namespace rlfc;
    if (n == 0)
        return RLFC_OK;
    if (!d_resid || !d_label || q > 7 || tau_err < 0) {
        set_error("rlfc_ks_search: invalid argument");
        return RLFC_E_INVALID_ARG;
    }
    if (n >= (1ull << 31)) {
        set_error("rlfc_ks_search: n must be below 2^31");
        return RLFC_E_RANGE;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    { TraceScope trace_("ks_search_kernel", st); ks_search_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(d_resid, (uint32_t)n, q, tau_err, lam_q8, d_label); }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? RLFC_OK : cuda_fail(e, "rlfc_ks_search");
}

RLFC_API int rlfc_ks_compact(const uint8_t *d_label, size_t n, uint32_t *d_index, uint32_t *d_count,
                             void *cuda_stream)
{
    using namespace rlfc;
    if (!d_count || (n && (!d_label || !d_index))) {
        set_error("rlfc_ks_compact: null argument");
        return RLFC_E_INVALID_ARG;
    }
    if (n >= (1ull << 31)) {
        set_error("rlfc_ks_compact: n must be below 2^31");
        return RLFC_E_RANGE;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (n == 0) {
        const cudaError_t e = cudaMemsetAsync(d_count, 0, 4, st);
        return e == cudaSuccess ? RLFC_OK : cuda_fail(e, "rlfc_ks_compact");
    }
    const uint32_t chunks = (uint32_t)((n + kChunk - 1) / kChunk);
    uint32_t *part = nullptr;
    cudaError_t e = cudaMallocAsync(&part, 4ull * chunks, st);
    if (e != cudaSuccess)
        return cuda_fail(e, "rlfc_ks_compact scratch");
    { TraceScope trace_("compact_count_kernel", st); compact_count_kernel<<<chunks, 1024, 0, st>>>(d_label, (uint32_t)n, part); }
    { TraceScope trace_("compact_write_kernel", st); compact_write_kernel<<<chunks, 1024, 0, st>>>(d_label, (uint32_t)n, part, d_index, d_count); }
    e = cudaGetLastError();
    cudaFreeAsync(part, st);
    return e == cudaSuccess ? RLFC_OK : cuda_fail(e, "rlfc_ks_compact");
}

RLFC_API int rlfc_ks_features(const int16_t *d_resid, const uint8_t *d_label, const uint32_t *d_index, size_t n,
                              uint16_t *d_x, uint8_t *d_label_out, void *cuda_stream)
{
    using namespace rlfc;
    if (n == 0)
        return RLFC_OK;
    if (!d_resid || !d_x) {
        set_error("rlfc_ks_features: null argument");
        return RLFC_E_INVALID_ARG;
    }
    if (n >= (1ull << 31)) {
        set_error("rlfc_ks_features: n must be below 2^31");
        return RLFC_E_RANGE;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    { TraceScope trace_("ks_features_kernel", st); ks_features_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(d_resid, d_label, d_index, (uint32_t)n, d_x, d_label_out); }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? RLFC_OK : cuda_fail(e, "rlfc_ks_features");
}

RLFC_API int rlfc_mlp_loss_grad(const uint16_t *d_w, const uint16_t *d_x, const uint8_t *d_label,
                                const uint32_t *d_order, size_t n, float *d_grad, float *d_loss, void *cuda_stream)
{
    using namespace rlfc;
    if (n == 0)
        return RLFC_OK;
    if (!d_w || !d_x || !d_label || !d_grad || !d_loss) {
        set_error("rlfc_mlp_loss_grad: null argument");
        return RLFC_E_INVALID_ARG;
    }
    if (n >= (1ull << 31)) {
        set_error("rlfc_mlp_loss_grad: n must be below 2^31");
        return RLFC_E_RANGE;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const size_t smem = kWBytes + sizeof(float) * (kTileFloats + kP);
    cudaError_t e = cudaFuncSetAttribute(mlp_loss_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return cuda_fail(e, "rlfc_mlp_loss_grad");
    { TraceScope trace_("mlp_loss_grad_kernel", st); mlp_loss_grad_kernel<<<net_grid((uint32_t)n, sm_count()), kThreads, smem, st>>>(d_w, d_x, d_label, d_order, (uint32_t)n, d_grad, d_loss); }
    e = cudaGetLastError();
    return e == cudaSuccess ? RLFC_OK : cuda_fail(e, "rlfc_mlp_loss_grad");
}

RLFC_API int rlfc_mlp_adam(float *d_master, uint16_t *d_w, float *d_grad, float *d_m, float *d_v, float lr,
                           float beta1, float beta2, float eps, float grad_scale, uint32_t step, void *cuda_stream)
{
    using namespace rlfc;
    if (!d_master || !d_w || !d_grad || !d_m || !d_v || step == 0) {
        set_error("rlfc_mlp_adam: null argument or step 0");
        return RLFC_E_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const float c1 = 1.0f - powf(beta1, (float)step), c2 = 1.0f - powf(beta2, (float)step);
    { TraceScope trace_("mlp_adam_kernel", st); mlp_adam_kernel<<<(kP + 255) / 256, 256, 0, st>>>(d_master, d_w, d_grad, d_m, d_v, lr, beta1, beta2, eps, grad_scale, c1, c2); }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? RLFC_OK : cuda_fail(e, "rlfc_mlp_adam");
}

RLFC_API int rlfc_mlp_predict(const uint16_t *d_w, const uint16_t *d_x, size_t n, const uint32_t *d_index,
                              uint8_t *d_label, void *cuda_stream)
{
    using namespace rlfc;
    if (n == 0)
        return RLFC_OK;
    if (!d_w || !d_x || !d_label) {
        set_error("rlfc_mlp_predict: null argument");
        return RLFC_E_INVALID_ARG;
    }
    if (n >= (1ull << 31)) {
        set_error("rlfc_mlp_predict: n must be below 2^31");
        return RLFC_E_RANGE;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const size_t smem = kWBytes + sizeof(float) * kPredWarpFloats * (kThreads / 32);
    cudaError_t e = cudaFuncSetAttribute(mlp_predict_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return cuda_fail(e, "rlfc_mlp_predict");
    // every CTA resident at once (the loop over sample groups is grid-strided)
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mlp_predict_kernel, kThreads, smem)) != cudaSuccess)
        return cuda_fail(e, "rlfc_mlp_predict");
    const uint32_t groups = (uint32_t)((n + 4 * (kThreads / 32) - 1) / (4 * (kThreads / 32)));
    const int grid = (int)std::max<uint32_t>(1, std::min<uint32_t>(groups, (uint32_t)(std::max(per_sm, 1) * sm_count())));
    { TraceScope trace_("mlp_predict_kernel", st); mlp_predict_kernel<<<grid, kThreads, smem, st>>>(d_w, d_x, (uint32_t)n, d_index, d_label); }
    e = cudaGetLastError();
    return e == cudaSuccess ? RLFC_OK : cuda_fail(e, "rlfc_mlp_predict");
}

}  // extern "C"

// The learned encoder aid: per-block (shift, mode) search, the 48 block
// statistics, and a 48 -> 64 -> 64 -> 112 perceptron with its training
// (forward, softmax cross-entropy, backward, Adam) and inference kernels.
//
// Numerics: parameters and inputs are stored in BF16; every product, sum and
// activation is FP32 (BF16 values widen exactly).  The network is small
// (14 576 parameters, layers 48 to 112 wide), so the kernels keep the
// transposed weights, the gradient accumulators and one tile of 32 samples'
// activations in shared memory and use the FP32 SIMT pipes.
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

struct NetSmem {
    float *w1t, *b1, *w2t, *b2, *w3t, *b3;   // transposed weights [in][out]
    float *x, *h1, *h2, *z, *d2, *d1;        // one tile of activations / deltas
};

__device__ __forceinline__ NetSmem carve(float *base)
{
    NetSmem m;
    m.w1t = base;
    m.b1 = m.w1t + NI * NH;
    m.w2t = m.b1 + NH;
    m.b2 = m.w2t + NH * NH;
    m.w3t = m.b2 + NH;
    m.b3 = m.w3t + NH * NO;
    m.x = m.b3 + NO;
    m.h1 = m.x + kTile * NI;
    m.h2 = m.h1 + kTile * NH;
    m.z = m.h2 + kTile * NH;
    m.d2 = m.z + kTile * NO;
    m.d1 = m.d2 + kTile * NH;
    return m;
}

constexpr int kNetFloats = kP + kTile * (NI + NH + NH + NO + NH + NH);

__device__ void load_weights(const uint16_t *w, const NetSmem &m)
{
    for (int i = threadIdx.x; i < NH * NI; i += blockDim.x) {
        const int j = i / NI, k = i % NI;
        m.w1t[k * NH + j] = bf(w[oW1 + i]);
    }
    for (int i = threadIdx.x; i < NH * NH; i += blockDim.x) {
        const int j = i / NH, k = i % NH;
        m.w2t[k * NH + j] = bf(w[oW2 + i]);
    }
    for (int i = threadIdx.x; i < NO * NH; i += blockDim.x) {
        const int j = i / NH, k = i % NH;
        m.w3t[k * NO + j] = bf(w[oW3 + i]);
    }
    for (int i = threadIdx.x; i < NH; i += blockDim.x) {
        m.b1[i] = bf(w[oB1 + i]);
        m.b2[i] = bf(w[oB2 + i]);
    }
    for (int i = threadIdx.x; i < NO; i += blockDim.x)
        m.b3[i] = bf(w[oB3 + i]);
}

// out[s][j] = act(b[j] + sum_k in[s][k] wt[k][j]) for the tile; J outputs
// per thread, kThreads / kTile threads per sample.
template <int K, int N, bool kRelu>
__device__ __forceinline__ void dense(const float *in, const float *wt, const float *b, float *out)
{
    constexpr int per = N * kTile / kThreads;
    const int s = threadIdx.x / (kThreads / kTile), j0 = (threadIdx.x % (kThreads / kTile)) * per;
    float acc[per];
#pragma unroll
    for (int m = 0; m < per; m++)
        acc[m] = b[j0 + m];
    for (int k = 0; k < K; k++) {
        const float v = in[s * K + k];
#pragma unroll
        for (int m = 0; m < per; m++)
            acc[m] = fmaf(v, wt[k * N + j0 + m], acc[m]);
    }
#pragma unroll
    for (int m = 0; m < per; m++)
        out[s * N + j0 + m] = kRelu ? fmaxf(acc[m], 0.0f) : acc[m];
}

// Tile of samples [t0, t0 + kTile) in `order` (or in index order): inputs and
// classes (-1 for missing / invalid ones).
__device__ __forceinline__ void load_tile(const uint16_t *x, const uint8_t *label, const uint32_t *order,
                                          uint32_t n, uint32_t t0, const NetSmem &m, int *s_cls)
{
    for (int i = threadIdx.x; i < kTile * NI; i += blockDim.x) {
        const uint32_t s = i / NI, f = i % NI, g = t0 + s;
        float v = 0.0f;
        if (g < n)
            v = bf(x[(size_t)(order ? order[g] : g) * NI + f]);
        m.x[i] = v;
    }
    if (s_cls && threadIdx.x < kTile) {
        const uint32_t g = t0 + threadIdx.x;
        int c = -1;
        if (g < n) {
            const uint32_t lab = label[order ? order[g] : g];
            if ((lab & 31u) < (uint32_t)kNumModes)
                c = (int)((lab >> 5) * kNumModes + (lab & 31u));
        }
        s_cls[threadIdx.x] = c;
    }
}

__device__ __forceinline__ void forward_tile(const NetSmem &m)
{
    dense<NI, NH, true>(m.x, m.w1t, m.b1, m.h1);
    __syncthreads();
    dense<NH, NH, true>(m.h1, m.w2t, m.b2, m.h2);
    __syncthreads();
    dense<NH, NO, false>(m.h2, m.w3t, m.b3, m.z);
    __syncthreads();
}

__global__ void __launch_bounds__(kThreads) mlp_loss_grad_kernel(const uint16_t *w, const uint16_t *x,
                                                                  const uint8_t *label, const uint32_t *order,
                                                                  uint32_t n, float *grad, float *loss)
{
    extern __shared__ __align__(16) float smem[];
    __shared__ int s_cls[kTile];
    __shared__ float s_loss;
    const NetSmem m = carve(smem);
    float *g = smem + kNetFloats;   // [kP] gradient accumulators, flat parameter order
    load_weights(w, m);
    for (int i = threadIdx.x; i < kP; i += blockDim.x)
        g[i] = 0.0f;
    if (threadIdx.x == 0)
        s_loss = 0.0f;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t ntiles = (n + kTile - 1) / kTile;
    for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        load_tile(x, label, order, n, t * kTile, m, s_cls);
        __syncthreads();
        forward_tile(m);
        // softmax cross-entropy; z becomes d loss / d z
        for (int s = warp; s < kTile; s += kThreads / 32) {
            float *z = m.z + s * NO;
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
        // layer 3: gW3[j][i] += sum_s dz[s][j] h2[s][i]; gb3; dh2 = dz W3 * relu'
        for (int e = threadIdx.x; e < NO * NH; e += kThreads) {
            const int j = e / NH, i = e % NH;
            float a = 0.0f;
            for (int s = 0; s < kTile; s++)
                a = fmaf(m.z[s * NO + j], m.h2[s * NH + i], a);
            g[oW3 + e] += a;
        }
        for (int j = threadIdx.x; j < NO; j += kThreads) {
            float a = 0.0f;
            for (int s = 0; s < kTile; s++)
                a += m.z[s * NO + j];
            g[oB3 + j] += a;
        }
        {
            const int s = threadIdx.x / 8, i0 = (threadIdx.x % 8) * 8;
            float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            for (int j = 0; j < NO; j++) {
                const float dz = m.z[s * NO + j];
#pragma unroll
                for (int u = 0; u < 8; u++)
                    acc[u] = fmaf(dz, m.w3t[(i0 + u) * NO + j], acc[u]);
            }
#pragma unroll
            for (int u = 0; u < 8; u++)
                m.d2[s * NH + i0 + u] = m.h2[s * NH + i0 + u] > 0.0f ? acc[u] : 0.0f;
        }
        __syncthreads();
        // layer 2
        for (int e = threadIdx.x; e < NH * NH; e += kThreads) {
            const int j = e / NH, i = e % NH;
            float a = 0.0f;
            for (int s = 0; s < kTile; s++)
                a = fmaf(m.d2[s * NH + j], m.h1[s * NH + i], a);
            g[oW2 + e] += a;
        }
        for (int j = threadIdx.x; j < NH; j += kThreads) {
            float a = 0.0f;
            for (int s = 0; s < kTile; s++)
                a += m.d2[s * NH + j];
            g[oB2 + j] += a;
        }
        {
            const int s = threadIdx.x / 8, i0 = (threadIdx.x % 8) * 8;
            float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            for (int j = 0; j < NH; j++) {
                const float d = m.d2[s * NH + j];
#pragma unroll
                for (int u = 0; u < 8; u++)
                    acc[u] = fmaf(d, m.w2t[(i0 + u) * NH + j], acc[u]);
            }
#pragma unroll
            for (int u = 0; u < 8; u++)
                m.d1[s * NH + i0 + u] = m.h1[s * NH + i0 + u] > 0.0f ? acc[u] : 0.0f;
        }
        __syncthreads();
        // layer 1
        for (int e = threadIdx.x; e < NH * NI; e += kThreads) {
            const int j = e / NI, i = e % NI;
            float a = 0.0f;
            for (int s = 0; s < kTile; s++)
                a = fmaf(m.d1[s * NH + j], m.x[s * NI + i], a);
            g[oW1 + e] += a;
        }
        for (int j = threadIdx.x; j < NH; j += kThreads) {
            float a = 0.0f;
            for (int s = 0; s < kTile; s++)
                a += m.d1[s * NH + j];
            g[oB1 + j] += a;
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < kP; i += blockDim.x)
        atomicAdd(&grad[i], g[i]);
    if (threadIdx.x == 0)
        atomicAdd(loss, s_loss);
}

// Inference, register blocked: each warp takes 4 samples at a time and lane l
// the outputs l, l + 32, ...; per input feature, one 16-byte broadcast of the
// 4 samples' activations and one weight per output feed 4 FMAs.  The
// activations of a warp's samples are its own columns of [feature][sample]
// arrays (row stride kRowT keeps the 16-byte stores on distinct banks), so the
// warps never wait on one another after the weights are loaded.
constexpr int kRowT = kTile + 4;

template <int K, int N, bool kRelu>
__device__ __forceinline__ void dense_cols(const float *inT, const float *wt, const float *b, int lane, int col,
                                           float acc[4][(N + 31) / 32])
{
    constexpr int kO = (N + 31) / 32;
#pragma unroll
    for (int i = 0; i < kO; i++) {
        const int o = lane + 32 * i;
        const float bias = o < N ? b[o] : 0.0f;
#pragma unroll
        for (int q = 0; q < 4; q++)
            acc[q][i] = bias;
    }
#pragma unroll 4
    for (int k = 0; k < K; k++) {
        const float4 v = *reinterpret_cast<const float4 *>(inT + k * kRowT + col);
#pragma unroll
        for (int i = 0; i < kO; i++) {
            const int o = lane + 32 * i;
            const float w = o < N ? wt[k * N + o] : 0.0f;
            acc[0][i] = fmaf(v.x, w, acc[0][i]);
            acc[1][i] = fmaf(v.y, w, acc[1][i]);
            acc[2][i] = fmaf(v.z, w, acc[2][i]);
            acc[3][i] = fmaf(v.w, w, acc[3][i]);
        }
    }
    if (kRelu) {
#pragma unroll
        for (int i = 0; i < kO; i++)
#pragma unroll
            for (int q = 0; q < 4; q++)
                acc[q][i] = fmaxf(acc[q][i], 0.0f);
    }
}

template <int N>
__device__ __forceinline__ void store_cols(float *outT, int lane, int col, const float acc[4][(N + 31) / 32])
{
#pragma unroll
    for (int i = 0; i < (N + 31) / 32; i++) {
        const int o = lane + 32 * i;
        if (o < N)
            *reinterpret_cast<float4 *>(outT + o * kRowT + col) = make_float4(acc[0][i], acc[1][i], acc[2][i], acc[3][i]);
    }
}

__global__ void __launch_bounds__(kThreads) mlp_predict_kernel(const uint16_t *w, const uint16_t *x, uint32_t n,
                                                                const uint32_t *index, uint8_t *label)
{
    extern __shared__ __align__(16) float smem[];
    const NetSmem m = carve(smem);
    float *xT = smem + kP, *h1T = xT + NI * kRowT, *h2T = h1T + NH * kRowT;
    load_weights(w, m);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, col = 4 * warp;
    const uint32_t ngroups = (n + 3) / 4;
    for (uint32_t grp = blockIdx.x * (kThreads / 32) + warp; grp < ngroups; grp += gridDim.x * (kThreads / 32)) {
        const uint32_t s0 = 4 * grp;
        for (int i = lane; i < 4 * NI; i += 32) {
            const int q = i / NI, f = i - q * NI;
            xT[f * kRowT + col + q] = s0 + q < n ? bf(x[(size_t)(s0 + q) * NI + f]) : 0.0f;
        }
        __syncwarp();
        {
            float a1[4][NH / 32];
            dense_cols<NI, NH, true>(xT, m.w1t, m.b1, lane, col, a1);
            store_cols<NH>(h1T, lane, col, a1);
        }
        __syncwarp();
        {
            float a2[4][NH / 32];
            dense_cols<NH, NH, true>(h1T, m.w2t, m.b2, lane, col, a2);
            store_cols<NH>(h2T, lane, col, a2);
        }
        __syncwarp();
        float z[4][(NO + 31) / 32];
        dense_cols<NH, NO, false>(h2T, m.w3t, m.b3, lane, col, z);
        // first maximum of each sample's logits over the lanes
#pragma unroll
        for (int q = 0; q < 4; q++) {
            float best = -INFINITY;
            int arg = 0;
#pragma unroll
            for (int i = 0; i < (NO + 31) / 32; i++) {
                const int o = lane + 32 * i;
                if (o < NO && z[q][i] > best) {
                    best = z[q][i];
                    arg = o;
                }
            }
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) {
                const float ob = __shfl_xor_sync(kFull, best, d);
                const int oa = __shfl_xor_sync(kFull, arg, d);
                if (ob > best || (ob == best && oa < arg)) {
                    best = ob;
                    arg = oa;
                }
            }
            const uint32_t gi = s0 + q;
            if (lane == 0 && gi < n)
                label[index ? index[gi] : gi] = (uint8_t)((arg % kNumModes) | (arg / kNumModes) << 5);
        }
        __syncwarp();   // the next group overwrites this warp's columns
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
    const size_t smem = sizeof(float) * (kNetFloats + kP);
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
    const size_t smem = sizeof(float) * (kP + (NI + 2 * NH) * kRowT);
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

/*
 * Oracle: the RLFC block decoder, Algorithm 2 -- TEST INFRASTRUCTURE ONLY.
 *
 *   Initialization: read the top RKVs, the block offsets and the SRV stream;
 *                   rebuild the BFS numbering of the tree (Section 3.5).
 *   DecompressLFIBlock(ImgIdx, BlkIdx):
 *     StartOffset <- BlockOffsets[BlkIdx]
 *     RKVBlock    <- the block of the view's top-level ancestor
 *     ParentIndx  <- the view's ancestor at every SRV level
 *     read and BISE-decode the ancestors' blocks, add them to RKVBlock
 *   then the inverse YCoCg-R gives RGB (Section 4).
 *
 * Readings: Algorithm 2 does not say which top RKV is read when there are
 * several; it is the view's top-level ancestor.  Channels are decoded
 * independently (Section 4, decode timings), one record per (location,
 * channel).  A dequantised value is (min + u) * 2^(q + s).  Colours outside
 * [0, 255] after the inverse transform (possible once residuals were
 * thresholded) are clamped.  Stopping before level 0 returns the filtered
 * value of that level (progressive decoding, Section 3.6).
 */
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

#define MAGIC 0x43464C52u
#define HDR_BITS 18

static uint32_t rd_u32(const uint8_t *p)
{
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}

static int rd_i16(const uint8_t *p)
{
    return (int)(int16_t)(uint16_t)((uint32_t)p[0] | ((uint32_t)p[1] << 8));
}

static long align16(long x) { return (x + 15) / 16 * 16; }

int or_stream_open(or_stream *s, const uint8_t *bytes, size_t nbytes)
{
    memset(s, 0, sizeof(*s));
    if (nbytes < 64 || rd_u32(bytes) != MAGIC || rd_u32(bytes + 4) != 1)
        return -1;
    s->bytes = bytes;
    s->nbytes = nbytes;
    s->U = (int)rd_u32(bytes + 8);
    s->V = (int)rd_u32(bytes + 12);
    s->W = (int)rd_u32(bytes + 16);
    s->H = (int)rd_u32(bytes + 20);
    s->B = (int)rd_u32(bytes + 24);
    s->L = (int)rd_u32(bytes + 28);
    s->q = (int)rd_u32(bytes + 32);
    s->n_top = (int)rd_u32(bytes + 36);
    s->S = (int)rd_u32(bytes + 40);
    s->off_top = rd_u32(bytes + 44);
    s->off_offsets = rd_u32(bytes + 48);
    s->off_records = rd_u32(bytes + 52);
    s->record_words = rd_u32(bytes + 56);
    if (s->U < 1 || s->V < 1 || s->W < 1 || s->H < 1 || s->B < 1 || s->B > 8 ||
        s->L < 2 || s->L > OR_MAXL || s->q > 7)
        return -1;
    if (64 + 8L * s->L > (long)nbytes)
        return -1;
    int Gu[OR_MAXL], Gv[OR_MAXL];
    long at = 64, nodes_total = 0;
    for (int l = 0; l < s->L; l++) {
        Gu[l] = (int)rd_u32(bytes + at);
        Gv[l] = (int)rd_u32(bytes + at + 4);
        at += 8;
        if (Gu[l] < 1 || Gv[l] < 1 || Gu[l] > 4096 || Gv[l] > 4096)
            return -1;
        if (l < s->L - 1)
            nodes_total += (long)Gu[l] * Gv[l];
    }
    if (Gu[0] != s->U || Gv[0] != s->V || at + 4 * nodes_total > s->off_top)
        return -1;
    int *par[OR_MAXL] = {0};
    for (int l = 0; l < s->L - 1; l++) {
        par[l] = malloc(sizeof(int) * Gu[l] * Gv[l]);
        for (int i = 0; i < Gu[l] * Gv[l]; i++) {
            par[l][i] = (int)rd_u32(bytes + at);
            at += 4;
        }
    }
    int rc = or_tree_from_parents(&s->tree, s->L, Gu, Gv, (const int *const *)par);
    for (int l = 0; l < OR_MAXL; l++)
        free(par[l]);
    if (rc != 0 || s->tree.n_top != s->n_top || s->tree.S != s->S)
        return -1;
    s->Wp = (s->W + s->B - 1) / s->B * s->B;
    s->Hp = (s->H + s->B - 1) / s->B * s->B;
    s->nlx = s->Wp / s->B;
    s->nly = s->Hp / s->B;
    s->nloc = s->nlx * s->nly;
    long top_bytes = 2L * s->n_top * 3 * s->Wp * s->Hp;
    if (s->off_top != align16(at) || s->off_offsets != align16(s->off_top + top_bytes) ||
        s->off_records != align16(s->off_offsets + 4 * (3L * s->nloc + 1)) ||
        (size_t)(s->off_records + 4 * s->record_words) != nbytes)
        return -1;
    uint32_t prev = 0;
    for (long i = 0; i <= 3L * s->nloc; i++) {
        uint32_t o = rd_u32(bytes + s->off_offsets + 4 * i);
        if (o < prev || o > (uint32_t)s->record_words || (i == 0 && o != 0))
            return -1;
        prev = o;
    }
    if (prev != (uint32_t)s->record_words)
        return -1;
    return 0;
}

void or_stream_close(or_stream *s)
{
    or_tree_free(&s->tree);
    memset(s, 0, sizeof(*s));
}

/* Adds node pos's block of record (loc, c) to acc; returns -1 on a corrupt
   record, 0 otherwise (an absent block adds nothing). */
static int add_srv_block(const or_stream *s, int loc, int c, int pos, int32_t *acc)
{
    const int n = s->B * s->B;
    const int MW = (s->S + 31) / 32;
    uint32_t w0 = rd_u32(s->bytes + s->off_offsets + 4 * (3L * loc + c));
    uint32_t w1 = rd_u32(s->bytes + s->off_offsets + 4 * (3L * loc + c + 1));
    const uint8_t *rec = s->bytes + s->off_records + 4L * w0;
    long rec_bits = 32L * (w1 - w0);
    if (rec_bits < 32L * MW)
        return -1;
    if (!or_get_bits(rec, pos, 1))
        return 0;
    int P = 0, rank = 0;
    for (int j = 0; j < s->S; j++) {
        if (or_get_bits(rec, j, 1)) {
            if (j < pos)
                rank++;
            P++;
        }
    }
    long hdr_pos = 32L * MW;
    long pay_pos = hdr_pos + (long)HDR_BITS * P;
    if (pay_pos > rec_bits)
        return -1;
    /* walk the present blocks before this one to find its payload */
    for (int r = 0; r < rank; r++) {
        int k = (int)or_get_bits(rec, hdr_pos + (long)HDR_BITS * r, 5);
        if (k >= OR_NMODES)
            return -1;
        pay_pos += or_bise_bits(n, k);
    }
    uint32_t hdr = or_get_bits(rec, hdr_pos + (long)HDR_BITS * rank, HDR_BITS);
    int k = (int)(hdr & 31u);
    int sh = (int)((hdr >> 5) & 3u);
    int mn = (int)((hdr >> 7) & 0x7FFu);
    if (mn >= 1024)
        mn -= 2048;
    if (k >= OR_NMODES || pay_pos + or_bise_bits(n, k) > rec_bits)
        return -1;
    int u[64];
    or_bise_unpack(rec, pay_pos, n, k, u);
    for (int i = 0; i < n; i++)
        acc[i] += (mn + u[i]) * (1 << (s->q + sh));
    return 0;
}

int or_decode_block_ycc(const or_stream *s, int view, int loc, int stop_level, int32_t *out)
{
    if (view < 0 || view >= s->U * s->V || loc < 0 || loc >= s->nloc ||
        stop_level < 0 || stop_level > s->L - 1)
        return -1;
    const int B = s->B, n = B * B;
    int anc[OR_MAXL];
    anc[0] = view;
    for (int l = 1; l < s->L; l++)
        anc[l] = s->tree.parent[l - 1][anc[l - 1]];
    int bx = loc % s->nlx, by = loc / s->nlx;
    long plane = (long)s->Wp * s->Hp;
    for (int c = 0; c < 3; c++) {
        int32_t *acc = out + c * n;
        /* ReadBlock(RKV^n, BlkIdx) */
        for (int i = 0; i < n; i++) {
            long idx = ((long)anc[s->L - 1] * 3 + c) * plane + (long)(by * B + i / B) * s->Wp + bx * B + i % B;
            acc[i] = rd_i16(s->bytes + s->off_top + 2 * idx);
        }
        /* ReadBlocks + BISEDecode + CombineBlocks, top level down */
        for (int l = s->L - 2; l >= stop_level; l--) {
            int pos = s->tree.pos_of[l][anc[l]];
            if (add_srv_block(s, loc, c, pos, acc) != 0)
                return -1;
        }
    }
    return 0;
}

static int clamp255(int v) { return v < 0 ? 0 : (v > 255 ? 255 : v); }

int or_decode_block(const or_stream *s, int view, int loc, uint8_t *out)
{
    const int n = s->B * s->B;
    int32_t ycc[3 * 64];
    if (or_decode_block_ycc(s, view, loc, 0, ycc) != 0)
        return -1;
    for (int i = 0; i < n; i++) {
        int r, g, b;
        or_ycocg_inv(ycc[i], ycc[n + i], ycc[2 * n + i], &r, &g, &b);
        out[3 * i] = (uint8_t)clamp255(r);
        out[3 * i + 1] = (uint8_t)clamp255(g);
        out[3 * i + 2] = (uint8_t)clamp255(b);
    }
    return 0;
}

int or_decode_all(const or_stream *s, uint8_t *out, int nthreads)
{
    const int B = s->B;
    const int nviews = s->U * s->V;
    int err = 0;
    if (nthreads < 1)
        nthreads = 1;
#pragma omp parallel for num_threads(nthreads) schedule(dynamic) reduction(| : err)
    for (int view = 0; view < nviews; view++) {
        uint8_t blk[64 * 3];
        for (int loc = 0; loc < s->nloc; loc++) {
            if (or_decode_block(s, view, loc, blk) != 0) {
                err |= 1;
                continue;
            }
            int bx = loc % s->nlx, by = loc / s->nlx;
            for (int i = 0; i < B * B; i++) {
                int x = bx * B + i % B, y = by * B + i / B;
                if (x >= s->W || y >= s->H)
                    continue;
                uint8_t *dst = out + (((long)view * s->H + y) * s->W + x) * 3;
                dst[0] = blk[3 * i];
                dst[1] = blk[3 * i + 1];
                dst[2] = blk[3 * i + 2];
            }
        }
    }
    return err ? -1 : 0;
}

/*
 * Oracle: the RLFC encoder, Algorithm 1 -- TEST INFRASTRUCTURE ONLY.
 *
 *   RKV^0 <- LFI (after YCoCg-R, Section 4)
 *   ComputeRKVTree: bottom-up clustering (Eq. 1) and weighted filtering (Eq. 2)
 *   ComputeSRVTree: top-down residuals (Eq. 3) with pixel thresholding, block
 *                   energy thresholding, quantisation and the recomputation of
 *                   each level from what was kept (Section 3.2)
 *   top-level RKVs stored losslessly (raw int16 in place of lossless JPEG2000)
 *   for each block location: gather the SRV blocks in BFS order (Section 3.4),
 *   BISE-encode them (Section 3.3), record the start offset (Fig. 4).
 *
 * Readings where the paper is silent (stream format v1):
 *  - Filter weights (Eq. 2): the paper says Gaussian-weighted and integer
 *    throughout.  A cluster of mu x mv nodes uses the binomial weights
 *    C(mu-1, a) * C(mv-1, b), the integer approximation of a Gaussian (a 2x2
 *    cluster is the plain four-image mean of Fig. 3), normalised by the power
 *    of two they sum to: RKV = floor((sum w X + 2^(s-1)) / 2^s),
 *    s = (mu-1) + (mv-1).
 *  - Thresholds: a residual is zeroed when |r| < tau_p; the block energy is the
 *    sum of |r| after that step and a block is dropped when it is below tau_b
 *    or zero.
 *  - Quantisation (the supplementary material is not available): a global
 *    shift q, qv = sign(r) * floor((|r| + h) / 2^q) with h = 2^(q-1) for q > 0
 *    (round half away from zero), reconstructed as qv * 2^q.  A kept block
 *    whose quantised values are all zero is dropped as well.
 *  - BISE range per block: min = min(qv) goes in the block header, the values
 *    qv - min are coded with the cheapest mode that holds their span.  With
 *    mode_space 1 each block instead gets the (mode, shift) of or_ks_search
 *    (ks.c), or a given one for the level-0 blocks, and is quantised with
 *    the global shift plus its own shift s (header bits 5..6).
 *  - Images whose side is not a multiple of B are padded by repeating the last
 *    column / row.
 *
 * Stream format v1 (little-endian):
 *   bytes 0..63  "RLFC", version 1, U, V, W, H, B, L, q, n_top, S, off_top,
 *                off_offsets, off_records, record_words, 0 (uint32 each);
 *   then the node grid (Gu, Gv) of every level, then the parent index of every
 *   node of levels 0..L-2;
 *   off_top: top RKVs, int16 [n_top][channel][Hp][Wp];
 *   off_offsets: 3 * nloc + 1 uint32, start word of record (loc, channel),
 *   then the total;
 *   off_records: per block location (row-major) and channel (Y, Co, Cg) a
 *   record: ceil(S/32) presence words (bit p = SRV node at BFS position p has
 *   a block), one 18-bit header per stored block (mode | shift << 5 |
 *   (min & 0x7FF) << 7), then the BISE payloads, padded to 32 bits.
 */
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

#define MAGIC 0x43464C52u /* bytes "RLFC" */
#define VERSION 1u
#define HDR_BITS 18

static long floor_div_pow2(long long a, int s)
{
    long long d = 1LL << s;
    long long qt = a / d;
    if ((a % d) != 0 && a < 0)
        qt -= 1;
    return (long)qt;
}

static long long binom(int m, int k)
{
    long long r = 1;
    for (int i = 1; i <= k; i++)
        r = r * (m - k + i) / i;
    return r;
}

/* Eq. 2 for one level: child holds Gu*Gv node images of npix samples each;
   parent_out receives ceil(Gu/c) * ceil(Gv/c) images. */
int or_filter_level(const int32_t *child, int Gu, int Gv, int c, int npix,
                    int32_t *parent_out)
{
    int ku = or_tile_count(Gu, c), kv = or_tile_count(Gv, c);
    for (int b = 0; b < kv; b++) {
        for (int a = 0; a < ku; a++) {
            int x0 = or_tile_lo(a, Gu, ku), x1 = or_tile_lo(a + 1, Gu, ku);
            int y0 = or_tile_lo(b, Gv, kv), y1 = or_tile_lo(b + 1, Gv, kv);
            int mu = x1 - x0, mv = y1 - y0;
            int s = (mu - 1) + (mv - 1);
            if (s > 60)
                return -1;
            long long half = s > 0 ? (1LL << (s - 1)) : 0;
            long long *w = malloc(sizeof(long long) * mu * mv);
            for (int y = y0; y < y1; y++)
                for (int x = x0; x < x1; x++)
                    w[(y - y0) * mu + (x - x0)] = binom(mu - 1, x - x0) * binom(mv - 1, y - y0);
            int32_t *dst = parent_out + (long)(b * ku + a) * npix;
            for (int i = 0; i < npix; i++) {
                long long acc = 0;
                for (int y = y0; y < y1; y++)
                    for (int x = x0; x < x1; x++)
                        acc += w[(y - y0) * mu + (x - x0)] * child[(long)(y * Gu + x) * npix + i];
                dst[i] = (int32_t)floor_div_pow2(acc + half, s);
            }
            free(w);
        }
    }
    return 0;
}

static void put_u32(uint8_t *p, uint32_t v)
{
    p[0] = (uint8_t)v;
    p[1] = (uint8_t)(v >> 8);
    p[2] = (uint8_t)(v >> 16);
    p[3] = (uint8_t)(v >> 24);
}

static void put_i16(uint8_t *p, int v)
{
    uint16_t u = (uint16_t)(int16_t)v;
    p[0] = (uint8_t)u;
    p[1] = (uint8_t)(u >> 8);
}

static long align16(long x) { return (x + 15) / 16 * 16; }

typedef struct {
    int n;            /* values per block */
    int S, MW;        /* SRV nodes, mask words */
} rec_shape;

int or_encode(const uint8_t *rgb, const or_params *p, uint8_t **out, size_t *nbytes)
{
    *out = NULL;
    *nbytes = 0;
    if (p->U < 1 || p->V < 1 || p->W < 1 || p->H < 1 || p->B < 1 || p->B > 8 ||
        p->L < 2 || p->L > OR_MAXL || p->tau_p < 0 || p->tau_b < 0 || p->q < 0 || p->q > 7 ||
        p->mode_space < 0 || p->mode_space > 1 || p->tau_err < 0 || p->lam_q8 < 0)
        return -1;
    const int U = p->U, V = p->V, W = p->W, H = p->H, B = p->B, L = p->L, q = p->q;
    const int n = B * B;
    const int Wp = (W + B - 1) / B * B, Hp = (H + B - 1) / B * B;
    const int nlx = Wp / B, nly = Hp / B, nloc = nlx * nly;
    const long plane = (long)Wp * Hp;   /* samples per channel plane */
    const long npix = 3 * plane;        /* samples per node image */

    or_tree tree;
    if (or_tree_from_clusters(&tree, U, V, L, p->c) != 0) {
        or_tree_free(&tree);
        return -1;
    }
    int nodes[OR_MAXL];
    for (int l = 0; l < L; l++)
        nodes[l] = tree.Gu[l] * tree.Gv[l];

    /* RKV^0: YCoCg-R of the padded views, stored as [node][channel][Hp][Wp] */
    int32_t *img[OR_MAXL] = {0};
    int32_t *rec[OR_MAXL] = {0};
    img[0] = malloc(sizeof(int32_t) * npix * nodes[0]);
    for (int vi = 0; vi < nodes[0]; vi++) {
        for (int y = 0; y < Hp; y++) {
            for (int x = 0; x < Wp; x++) {
                int sx = x < W ? x : W - 1, sy = y < H ? y : H - 1;
                const uint8_t *px = rgb + (((long)vi * H + sy) * W + sx) * 3;
                int yy, co, cg;
                or_ycocg_fwd(px[0], px[1], px[2], &yy, &co, &cg);
                int32_t *dst = img[0] + (long)vi * npix;
                dst[0 * plane + (long)y * Wp + x] = yy;
                dst[1 * plane + (long)y * Wp + x] = co;
                dst[2 * plane + (long)y * Wp + x] = cg;
            }
        }
    }

    /* ComputeRKVTree (Eq. 1-2), bottom-up */
    for (int l = 1; l < L; l++) {
        img[l] = malloc(sizeof(int32_t) * npix * nodes[l]);
        or_filter_level(img[l - 1], tree.Gu[l - 1], tree.Gv[l - 1], p->c[l], (int)npix, img[l]);
    }

    /* ComputeSRVTree (Eq. 3), top-down with recomputation.  The quantised SRV
       of a node replaces its RKV image in img[] once used; present[] marks the
       kept blocks.  rec[l] is the recomputed level l (rec[L-1] = top RKVs). */
    unsigned char *present[OR_MAXL] = {0};
    unsigned char *kmode[OR_MAXL] = {0};   /* per stored block: k | s << 5 */
    int srv_err = 0;
    rec[L - 1] = malloc(sizeof(int32_t) * npix * nodes[L - 1]);
    memcpy(rec[L - 1], img[L - 1], sizeof(int32_t) * npix * nodes[L - 1]);
    const int half = q > 0 ? 1 << (q - 1) : 0;
    int *r = malloc(sizeof(int) * n);
    int *qv = malloc(sizeof(int) * n);
    for (int l = L - 1; l >= 1; l--) {
        int lc = l - 1;
        present[lc] = calloc((size_t)nodes[lc] * 3 * nloc, 1);
        kmode[lc] = calloc((size_t)nodes[lc] * 3 * nloc, 1);
        if (lc >= 1)
            rec[lc] = malloc(sizeof(int32_t) * npix * nodes[lc]);
        for (int x = 0; x < nodes[lc]; x++) {
            int par = tree.parent[lc][x];
            for (int c = 0; c < 3; c++) {
                for (int b = 0; b < nloc; b++) {
                    int bx = b % nlx, by = b / nlx;
                    long energy = 0;
                    for (int k = 0; k < n; k++) {
                        long at = c * plane + (long)(by * B + k / B) * Wp + bx * B + k % B;
                        int resid = img[lc][(long)x * npix + at] - rec[l][(long)par * npix + at];
                        if (resid < p->tau_p && -resid < p->tau_p)
                            resid = 0;
                        r[k] = resid;
                        energy += resid < 0 ? -resid : resid;
                    }
                    int keep = energy > 0 && energy >= p->tau_b;
                    const long bi = ((long)x * 3 + c) * nloc + b;
                    int ks_k = 0, ks_s = 0, have = 0;
                    if (lc == 0 && p->leaf_resid)
                        for (int k = 0; k < n; k++)
                            p->leaf_resid[bi * n + k] = (int16_t)r[k];
                    if (lc == 0 && p->leaf_label) {
                        int lk, ls;
                        p->leaf_label[bi] = keep && or_ks_search(r, n, q, p->tau_err, p->lam_q8, &lk, &ls) == 0
                                                ? (uint8_t)(lk | ls << 5) : 0xFF;
                    }
                    if (keep && p->mode_space == 1) {
                        /* a given leaf mode is used when it is a candidate */
                        if (lc == 0 && p->leaf_modes && p->leaf_modes[bi] != 0xFF) {
                            long long cost;
                            int gk = p->leaf_modes[bi] & 31, gs = p->leaf_modes[bi] >> 5;
                            if (or_ks_cost(r, n, q, gs, gk, p->tau_err, p->lam_q8, &cost) == 0) {
                                ks_k = gk;
                                ks_s = gs;
                                have = 1;
                            }
                        }
                        if (!have && or_ks_search(r, n, q, p->tau_err, p->lam_q8, &ks_k, &ks_s) != 0)
                            srv_err = 1;
                    }
                    const int t = q + ks_s;
                    const int ht = t > 0 ? 1 << (t - 1) : 0;
                    int nonzero = 0;
                    for (int k = 0; k < n; k++) {
                        int mag = r[k] < 0 ? -r[k] : r[k];
                        int qm = (mag + (p->mode_space == 1 ? ht : half)) >> (p->mode_space == 1 ? t : q);
                        qv[k] = keep ? (r[k] < 0 ? -qm : qm) : 0;
                        if (qv[k] != 0)
                            nonzero = 1;
                    }
                    if (!nonzero)
                        keep = 0;
                    if (keep && p->mode_space == 0) {
                        int mn = qv[0], mx = qv[0];
                        for (int k = 1; k < n; k++) {
                            if (qv[k] < mn) mn = qv[k];
                            if (qv[k] > mx) mx = qv[k];
                        }
                        ks_k = or_choose_mode_search(n, mx - mn);
                        if (ks_k < 0)
                            srv_err = 1;
                    }
                    present[lc][bi] = (unsigned char)keep;
                    kmode[lc][bi] = (unsigned char)(keep ? (ks_k | ks_s << 5) : 0);
                    for (int k = 0; k < n; k++) {
                        long at = c * plane + (long)(by * B + k / B) * Wp + bx * B + k % B;
                        int add = keep ? qv[k] * (1 << (q + ks_s)) : 0;
                        if (lc >= 1)
                            rec[lc][(long)x * npix + at] = rec[l][(long)par * npix + at] + add;
                        img[lc][(long)x * npix + at] = keep ? qv[k] : 0;
                    }
                }
            }
        }
    }

    /* Stream assembly (Algorithm 1, Fig. 4) */
    const int S = tree.S, MW = (S + 31) / 32;
    long hdr_bytes = 64 + 8L * L;
    for (int l = 0; l < L - 1; l++)
        hdr_bytes += 4L * nodes[l];
    const long off_top = align16(hdr_bytes);
    const long top_bytes = 2L * nodes[L - 1] * npix;
    const long off_offsets = align16(off_top + top_bytes);
    const long n_offsets = 3L * nloc + 1;
    const long off_records = align16(off_offsets + 4 * n_offsets);

    /* pass 1: the length of every record */
    long *rec_words = malloc(sizeof(long) * 3 * nloc);
    int *u = malloc(sizeof(int) * n);
    int err = srv_err;
    long total_words = 0;
    for (int b = 0; b < nloc && !err; b++) {
        int bx = b % nlx, by = b / nlx;
        for (int c = 0; c < 3; c++) {
            long bits = 32L * MW;
            for (int pos = 0; pos < S; pos++) {
                int lv = tree.bfs_level[pos], nd = tree.bfs_node[pos];
                if (!present[lv][((long)nd * 3 + c) * nloc + b])
                    continue;
                int mn = 0, mx = 0;
                for (int k = 0; k < n; k++) {
                    long at = c * plane + (long)(by * B + k / B) * Wp + bx * B + k % B;
                    int v = img[lv][(long)nd * npix + at];
                    if (k == 0 || v < mn) mn = v;
                    if (k == 0 || v > mx) mx = v;
                }
                int mode = kmode[lv][((long)nd * 3 + c) * nloc + b] & 31;
                if (or_mode_N(mode) < mx - mn + 1 || mn < -1024 || mn > 1023) {
                    err = 1;
                    break;
                }
                bits += HDR_BITS + or_bise_bits(n, mode);
            }
            rec_words[3L * b + c] = (bits + 31) / 32;
            total_words += rec_words[3L * b + c];
        }
    }

    size_t total = (size_t)(off_records + 4 * total_words);
    uint8_t *buf = err ? NULL : calloc(total, 1);
    if (buf) {
        put_u32(buf + 0, MAGIC);
        put_u32(buf + 4, VERSION);
        put_u32(buf + 8, (uint32_t)U);
        put_u32(buf + 12, (uint32_t)V);
        put_u32(buf + 16, (uint32_t)W);
        put_u32(buf + 20, (uint32_t)H);
        put_u32(buf + 24, (uint32_t)B);
        put_u32(buf + 28, (uint32_t)L);
        put_u32(buf + 32, (uint32_t)q);
        put_u32(buf + 36, (uint32_t)nodes[L - 1]);
        put_u32(buf + 40, (uint32_t)S);
        put_u32(buf + 44, (uint32_t)off_top);
        put_u32(buf + 48, (uint32_t)off_offsets);
        put_u32(buf + 52, (uint32_t)off_records);
        put_u32(buf + 56, (uint32_t)total_words);
        put_u32(buf + 60, 0);
        long at = 64;
        for (int l = 0; l < L; l++) {
            put_u32(buf + at, (uint32_t)tree.Gu[l]);
            put_u32(buf + at + 4, (uint32_t)tree.Gv[l]);
            at += 8;
        }
        for (int l = 0; l < L - 1; l++)
            for (int i = 0; i < nodes[l]; i++) {
                put_u32(buf + at, (uint32_t)tree.parent[l][i]);
                at += 4;
            }
        /* top RKVs, lossless: [n_top][channel][Hp][Wp] int16 */
        for (long i = 0; i < (long)nodes[L - 1] * npix; i++)
            put_i16(buf + off_top + 2 * i, img[L - 1][i]);
        /* offsets: start word of every record, then the total */
        long w = 0;
        for (long i = 0; i < 3L * nloc; i++) {
            put_u32(buf + off_offsets + 4 * i, (uint32_t)w);
            w += rec_words[i];
        }
        put_u32(buf + off_offsets + 4 * (3L * nloc), (uint32_t)w);

        /* pass 2: the records */
        w = 0;
        for (int b = 0; b < nloc; b++) {
            int bx = b % nlx, by = b / nlx;
            for (int c = 0; c < 3; c++) {
                uint8_t *recp = buf + off_records + 4 * w;
                int P = 0;
                for (int pos = 0; pos < S; pos++) {
                    int lv = tree.bfs_level[pos], nd = tree.bfs_node[pos];
                    if (present[lv][((long)nd * 3 + c) * nloc + b]) {
                        or_put_bits(recp, pos, 1, 1u);
                        P++;
                    }
                }
                long hdr_pos = 32L * MW;
                long pay_pos = hdr_pos + (long)HDR_BITS * P;
                for (int pos = 0; pos < S; pos++) {
                    int lv = tree.bfs_level[pos], nd = tree.bfs_node[pos];
                    if (!present[lv][((long)nd * 3 + c) * nloc + b])
                        continue;
                    int mn = 0, mx = 0;
                    for (int k = 0; k < n; k++) {
                        long a2 = c * plane + (long)(by * B + k / B) * Wp + bx * B + k % B;
                        int v = img[lv][(long)nd * npix + a2];
                        if (k == 0 || v < mn) mn = v;
                        if (k == 0 || v > mx) mx = v;
                        u[k] = v;
                    }
                    for (int k = 0; k < n; k++)
                        u[k] -= mn;
                    const int km = kmode[lv][((long)nd * 3 + c) * nloc + b];
                    int mode = km & 31;
                    uint32_t header = (uint32_t)mode | ((uint32_t)(km >> 5) << 5) | (((uint32_t)mn & 0x7FFu) << 7);
                    or_put_bits(recp, hdr_pos, HDR_BITS, header);
                    hdr_pos += HDR_BITS;
                    or_bise_pack(recp, pay_pos, n, mode, u);
                    pay_pos += or_bise_bits(n, mode);
                }
                w += rec_words[3L * b + c];
            }
        }
        *out = buf;
        *nbytes = total;
    }

    free(u);
    free(rec_words);
    free(r);
    free(qv);
    for (int l = 0; l < OR_MAXL; l++) {
        free(img[l]);
        free(rec[l]);
        free(present[l]);
        free(kmode[l]);
    }
    or_tree_free(&tree);
    return buf ? 0 : -1;
}

void or_free(void *ptr)
{
    free(ptr);
}

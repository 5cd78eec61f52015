/*
 * RLFC CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, deliberately unoptimised restatement of the RLFC method
 * (Pratapa & Manocha, "RLFC: Random Access Light Field Compression using Key
 * Views and Bounded Integer Sequence Encoding", I3D 2019).  It exists so that
 * the CUDA library can be checked against something written straight from the
 * paper.  Only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load it; the product library never links or calls it, and it
 * shares no code, header, table or helper with the product library.
 *
 * Every function names the passage of the paper it follows.  Where the paper
 * is silent the oracle takes the reading written next to the function; the
 * byte layout of the stream ("stream format v1") is stated in encode.c.
 *
 * Parity status: every function here is pinned by a CPU test against a closed
 * form, an exhaustive or brute-force check, a library routine or a stated
 * invariant, except the bpp/PSNR figures of the paper's Tables 1-3, which need
 * datasets that are not available ("parity unpinned" for those numbers only).
 */
#ifndef RLFC_ORACLE_H
#define RLFC_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OR_NMODES 28
#define OR_MAXL 8

/* ---- colour.c : lossless YCoCg-R (Section 4, Malvar & Sullivan lifting) ---- */
void or_ycocg_fwd(int r, int g, int b, int *y, int *co, int *cg);
void or_ycocg_inv(int y, int co, int cg, int *r, int *g, int *b);
/* rgb: npx*3 bytes; out: npx*3 ints (Y, Co, Cg per pixel) */
void or_ycocg_fwd_array(const uint8_t *rgb, long npx, int32_t *out);
/* ycc: npx*3 ints; out: npx*3 ints (R, G, B, not clamped) */
void or_ycocg_inv_array(const int32_t *ycc, long npx, int32_t *out);

/* ---- bise.c : bounded integer sequence encoding (Section 3.3) ---- */
int or_mode_N(int k);    /* value range N of mode k (0..27), ascending in k */
int or_mode_kind(int k); /* 0 = plain bits, 1 = trits, 2 = quints */
int or_mode_b(int k);    /* low bits per value */
long or_bise_bits(int n, int k);          /* packed length of n values */
int or_choose_mode_search(int n, int span);  /* exhaustive min-cost search */
void or_put_bits(uint8_t *buf, long pos, int width, uint32_t value);
uint32_t or_get_bits(const uint8_t *buf, long pos, int width);
/* pack n values u[i] < N_k starting at bit pos of a zeroed buffer */
void or_bise_pack(uint8_t *buf, long pos, int n, int k, const int *u);
void or_bise_unpack(const uint8_t *buf, long pos, int n, int k, int *u);
long or_bise_exhaustive(int n, int k, long max_count);

/* ---- tree.c : clusters (Eq. 1) and the BFS linearisation (Section 3.4) ---- */
typedef struct {
    int L;                 /* number of levels; level 0 = the input views */
    int Gu[OR_MAXL], Gv[OR_MAXL];
    int *parent[OR_MAXL];  /* parent[l][node] = node index at level l+1, l < L-1 */
    int n_top;             /* nodes at level L-1 (top RKVs) */
    int S;                 /* SRV nodes = nodes at levels 0..L-2 */
    int *bfs_level;        /* [S] level of the SRV node at BFS position p */
    int *bfs_node;         /* [S] node index of the SRV node at BFS position p */
    int *pos_of[OR_MAXL];  /* pos_of[l][node] = BFS position, l < L-1 */
} or_tree;

int or_tile_count(int G, int c);
int or_tile_lo(int a, int G, int k);
int or_tree_from_clusters(or_tree *t, int U, int V, int L, const int *c);
int or_tree_from_parents(or_tree *t, int L, const int *Gu, const int *Gv,
                         const int *const *parent);
void or_tree_free(or_tree *t);

/* ---- encode.c : Algorithm 1 with Eq. 2 (filter) and Eq. 3 (residuals) ---- */
typedef struct {
    int U, V, W, H;        /* view grid and view size */
    int B;                 /* block side; n = B*B values per channel block */
    int L;                 /* tree levels (>= 2) */
    int c[OR_MAXL];        /* cluster side per level, c[1..L-1] */
    int tau_p;             /* pixel threshold: |r| < tau_p -> 0 */
    int tau_b;             /* block energy threshold: sum|r| < tau_b -> dropped */
    int q;                 /* global quantisation shift */
    /* block modes: 0 = plain method (s = 0, cheapest range); 1 = per-block
       (mode, shift) by or_ks_search, or taken from leaf_modes when given */
    int mode_space;
    int tau_err;           /* largest error a shift s > 0 may add */
    int lam_q8;            /* distortion weight of the search, 1/256 bits per squared error */
    const uint8_t *leaf_modes;  /* optional [U*V][3][nloc]: k | s << 5 for the level-0
                                   blocks, 0xFF = search; an infeasible entry falls back
                                   to the search (mode_space 1 only) */
    int16_t *leaf_resid;   /* optional out [U*V][3][nloc][n]: level-0 residuals after the
                              pixel threshold */
    uint8_t *leaf_label;   /* optional out [U*V][3][nloc]: or_ks_search's k | s << 5 for the
                              level-0 blocks kept by the energy test, 0xFF for the others */
} or_params;

/* rgb: [V][U][H][W][3].  On success *out is malloc'ed; release with or_free. */
int or_encode(const uint8_t *rgb, const or_params *p, uint8_t **out, size_t *nbytes);
void or_free(void *ptr);
/* binomial cluster filter of one level (Eq. 2), exposed for tests */
int or_filter_level(const int32_t *child, int Gu, int Gv, int c, int npix,
                    int32_t *parent_out);

/* ---- ks.c : per-block (mode, shift) search of the learned encoder aid ---- */
void or_ks_quantise(const int *r, int n, int q, int s, int *qv);
/* 0 and *cost = 256 * bits + lam_q8 * SSE when (s, k) is a candidate, else -1 */
int or_ks_cost(const int *r, int n, int q, int s, int k, int tau_err, int lam_q8, long long *cost);
int or_ks_search(const int *r, int n, int q, int tau_err, int lam_q8, int *k_out, int *s_out);
/* the 48 statistics of a 16-value block, in the network's input order */
void or_ks_features(const int *r, double *f);

/* ---- mlp.c : the aid's network, 48 -> 64 -> 64 -> 112, FP64 ---- */
int or_mlp_nparams(void);
void or_mlp_forward(const double *w, const double *x, int n, double *logits);
int or_mlp_loss_grad(const double *w, const double *x, const int *y, int n, double *grad, double *loss);

/* ---- decode.c : Algorithm 2 ---- */
typedef struct {
    const uint8_t *bytes;
    size_t nbytes;
    int U, V, W, H, B, L, q, n_top, S;
    int Wp, Hp, nlx, nly, nloc;
    long off_top, off_offsets, off_records, record_words;
    or_tree tree;
} or_stream;

int or_stream_open(or_stream *s, const uint8_t *bytes, size_t nbytes);
void or_stream_close(or_stream *s);
/* decode one block: out = B*B*3 bytes, row-major pixels, RGB */
int or_decode_block(const or_stream *s, int view, int loc, uint8_t *out);
/* decode one block in YCoCg-R before the colour inverse: out = 3*B*B ints,
   channel-major; levels_used < L-1 stops the traversal early (Section 3.6) */
int or_decode_block_ycc(const or_stream *s, int view, int loc, int stop_level,
                        int32_t *out);
/* decode every view: out = [V*U][H][W][3] (cropped to W x H) */
int or_decode_all(const or_stream *s, uint8_t *out, int nthreads);

/* ---- render.c : new-view interpolation (Section 3.6), FP64 ---- */
/* lf: decoded views [V*U][H][W][3]; writes out[3] in [0,1] */
void or_render_pixel(const uint8_t *lf, int U, int V, int W, int H,
                     double u, double v, double d, int out_w, int out_h,
                     int x, int y, double *out);
void or_render_view(const uint8_t *lf, int U, int V, int W, int H,
                    double u, double v, double d, int out_w, int out_h,
                    double *out);

#ifdef __cplusplus
}
#endif
#endif

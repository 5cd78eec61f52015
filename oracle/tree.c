/*
 * Oracle: the RKV/SRV tree shape and its BFS linearisation -- TEST
 * INFRASTRUCTURE ONLY.
 *
 * Eq. 1 groups spatially close views of level l-1 into clusters whose RKV is
 * a node of level l.  The paper only says "dist < threshold" and that the
 * first level uses clusters of four neighbouring views (Fig. 3); the reading
 * here is a uniform tiling of the level's (u, v) grid: with cluster side c an
 * axis of G nodes is cut into k = ceil(G / c) tiles, tile a covering
 * [floor(a G / k), floor((a + 1) G / k)).  Node index at a level is row-major,
 * y * Gu + x (x along u).
 *
 * Section 3.4: the final tree is linearised by breadth-first search from the
 * root; every SRV block inherits its node's serial index.  With more than one
 * top RKV the search starts from all of them in index order; children are
 * visited in increasing node index.  BFS positions count SRV nodes only (the
 * top RKVs are stored separately), so position 0 is the first node of level
 * L-2.  Section 3.5 recomputes the same search when decoding starts.
 */
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

int or_tile_count(int G, int c)
{
    return (G + c - 1) / c;
}

int or_tile_lo(int a, int G, int k)
{
    return (int)(((long)a * G) / k);
}

static int tile_of(int x, int G, int k)
{
    for (int a = 0; a < k; a++)
        if (or_tile_lo(a, G, k) <= x && x < or_tile_lo(a + 1, G, k))
            return a;
    return -1;
}

static int bfs(or_tree *t)
{
    int L = t->L;
    int total = 0;
    for (int l = 0; l < L; l++)
        total += t->Gu[l] * t->Gv[l];
    t->n_top = t->Gu[L - 1] * t->Gv[L - 1];
    t->S = total - t->n_top;
    int *ql = malloc(sizeof(int) * total);
    int *qn = malloc(sizeof(int) * total);
    t->bfs_level = malloc(sizeof(int) * (t->S > 0 ? t->S : 1));
    t->bfs_node = malloc(sizeof(int) * (t->S > 0 ? t->S : 1));
    for (int l = 0; l < L - 1; l++) {
        t->pos_of[l] = malloc(sizeof(int) * t->Gu[l] * t->Gv[l]);
        for (int i = 0; i < t->Gu[l] * t->Gv[l]; i++)
            t->pos_of[l][i] = -1;
    }
    int head = 0, tail = 0, pos = 0;
    for (int i = 0; i < t->n_top; i++) {
        ql[tail] = L - 1;
        qn[tail] = i;
        tail++;
    }
    while (head < tail) {
        int lv = ql[head], nd = qn[head];
        head++;
        if (lv < L - 1) {
            t->bfs_level[pos] = lv;
            t->bfs_node[pos] = nd;
            t->pos_of[lv][nd] = pos;
            pos++;
        }
        if (lv > 0) {
            int nchild = t->Gu[lv - 1] * t->Gv[lv - 1];
            for (int ch = 0; ch < nchild; ch++) {
                if (t->parent[lv - 1][ch] == nd) {
                    ql[tail] = lv - 1;
                    qn[tail] = ch;
                    tail++;
                }
            }
        }
    }
    free(ql);
    free(qn);
    /* every SRV node must be reachable from a top node */
    return pos == t->S ? 0 : -1;
}

int or_tree_from_clusters(or_tree *t, int U, int V, int L, const int *c)
{
    memset(t, 0, sizeof(*t));
    if (L < 2 || L > OR_MAXL || U < 1 || V < 1)
        return -1;
    t->L = L;
    t->Gu[0] = U;
    t->Gv[0] = V;
    for (int l = 1; l < L; l++) {
        if (c[l] < 1)
            return -1;
        t->Gu[l] = or_tile_count(t->Gu[l - 1], c[l]);
        t->Gv[l] = or_tile_count(t->Gv[l - 1], c[l]);
    }
    for (int l = 0; l < L - 1; l++) {
        int Gu = t->Gu[l], Gv = t->Gv[l];
        int ku = t->Gu[l + 1], kv = t->Gv[l + 1];
        t->parent[l] = malloc(sizeof(int) * Gu * Gv);
        for (int y = 0; y < Gv; y++)
            for (int x = 0; x < Gu; x++)
                t->parent[l][y * Gu + x] = tile_of(y, Gv, kv) * ku + tile_of(x, Gu, ku);
    }
    return bfs(t);
}

int or_tree_from_parents(or_tree *t, int L, const int *Gu, const int *Gv,
                         const int *const *parent)
{
    memset(t, 0, sizeof(*t));
    if (L < 2 || L > OR_MAXL)
        return -1;
    t->L = L;
    for (int l = 0; l < L; l++) {
        if (Gu[l] < 1 || Gv[l] < 1)
            return -1;
        t->Gu[l] = Gu[l];
        t->Gv[l] = Gv[l];
    }
    for (int l = 0; l < L - 1; l++) {
        int n = Gu[l] * Gv[l], np = Gu[l + 1] * Gv[l + 1];
        t->parent[l] = malloc(sizeof(int) * n);
        for (int i = 0; i < n; i++) {
            if (parent[l][i] < 0 || parent[l][i] >= np)
                return -1;
            t->parent[l][i] = parent[l][i];
        }
    }
    return bfs(t);
}

void or_tree_free(or_tree *t)
{
    for (int l = 0; l < OR_MAXL; l++) {
        free(t->parent[l]);
        free(t->pos_of[l]);
    }
    free(t->bfs_level);
    free(t->bfs_node);
    memset(t, 0, sizeof(*t));
}

/*
 * Oracle: the (mode, shift) search of the learned encoder aid -- TEST
 * INFRASTRUCTURE ONLY.
 *
 * The block header of stream format v1 carries a 2-bit per-block shift s
 * beside the 5-bit BISE mode k (Section 3.3 codes each block with its own
 * range; the shift is an extension of that choice, the paper has none).  A kept block's
 * residuals r are then stored as qv = sign(r) floor((|r| + h) / 2^(q+s)),
 * h = 2^(q+s-1) (none when q+s = 0), and reconstructed as qv 2^(q+s): a larger
 * shift shrinks the range to code at the price of distortion.
 *
 * The search is the plain exhaustive definition: every (s, k) with s in 0..3
 * and k in 0..27 whose range N_k holds span(qv_s) + 1 values, and, for s > 0,
 * whose largest error max |r - qv_s 2^(q+s)| is at most tau_err, is a
 * candidate; the cost is 256 * payload bits + lam_q8 * SSE (an integer, so
 * every implementation takes the same decision); the first candidate of least
 * cost in (s, k) order wins.  s = 0 is the plain method and is always a
 * candidate when its span fits the largest mode.
 *
 * The 48 block statistics fed to the network are defined here as well
 * (or_ks_features).
 */
#include <math.h>
#include <stdlib.h>

#include "oracle.h"

void or_ks_quantise(const int *r, int n, int q, int s, int *qv)
{
    const int t = q + s;
    const int h = t > 0 ? 1 << (t - 1) : 0;
    for (int i = 0; i < n; i++) {
        int mag = r[i] < 0 ? -r[i] : r[i];
        int m = (mag + h) >> t;
        qv[i] = r[i] < 0 ? -m : m;
    }
}

int or_ks_cost(const int *r, int n, int q, int s, int k, int tau_err, int lam_q8, long long *cost)
{
    int qv[64];
    if (n > 64 || k < 0 || k >= OR_NMODES || s < 0 || s > 3)
        return -1;
    or_ks_quantise(r, n, q, s, qv);
    int mn = qv[0], mx = qv[0];
    long long sse = 0;
    int maxerr = 0;
    for (int i = 0; i < n; i++) {
        if (qv[i] < mn) mn = qv[i];
        if (qv[i] > mx) mx = qv[i];
        int e = r[i] - qv[i] * (1 << (q + s));
        if (e < 0) e = -e;
        if (e > maxerr) maxerr = e;
        sse += (long long)e * e;
    }
    if (or_mode_N(k) < mx - mn + 1 || mn < -1024 || mn > 1023)
        return -1;
    if (s > 0 && maxerr > tau_err)
        return -1;
    *cost = 256LL * or_bise_bits(n, k) + (long long)lam_q8 * sse;
    return 0;
}

int or_ks_search(const int *r, int n, int q, int tau_err, int lam_q8, int *k_out, int *s_out)
{
    long long best = 0;
    int found = 0;
    for (int s = 0; s < 4; s++) {
        for (int k = 0; k < OR_NMODES; k++) {
            long long c;
            if (or_ks_cost(r, n, q, s, k, tau_err, lam_q8, &c) != 0)
                continue;
            if (!found || c < best) {
                best = c;
                *k_out = k;
                *s_out = s;
                found = 1;
            }
        }
    }
    return found ? 0 : -1;
}

static int cmp_int(const void *a, const void *b)
{
    int x = *(const int *)a, y = *(const int *)b;
    return (x > y) - (x < y);
}

/*
 * The 48 statistics of a 16-value residual block (scaled to about unit size):
 *   f[0..15]  the values sorted ascending / 32
 *   f[16..31] the values in raster order / 32
 *   f[32] mean / 32        f[33] standard deviation / 32
 *   f[34] min / 32         f[35] max / 32
 *   f[36] span / 64        f[37] max |r| / 32
 *   f[38] sum |r| / 256    f[39] non-zero values / 16
 *   f[40] odd values / 16  f[41] values = 2 (mod 4) / 16
 *   f[42] values = 4 (mod 8) / 16
 *   f[43..46] values with |r| <= 1, 2, 4, 8, each / 16
 *   f[47] log2(span + 1) / 10
 */
void or_ks_features(const int *r, double *f)
{
    int s[16];
    double sum = 0.0, sum2 = 0.0, l1 = 0.0;
    int mn = r[0], mx = r[0], amax = 0, nz = 0, odd = 0, m4 = 0, m8 = 0, le[4] = {0, 0, 0, 0};
    for (int i = 0; i < 16; i++) {
        s[i] = r[i];
        int a = r[i] < 0 ? -r[i] : r[i];
        sum += r[i];
        sum2 += (double)r[i] * r[i];
        l1 += a;
        if (r[i] < mn) mn = r[i];
        if (r[i] > mx) mx = r[i];
        if (a > amax) amax = a;
        nz += r[i] != 0;
        odd += (a & 1) != 0;
        m4 += (a & 3) == 2;
        m8 += (a & 7) == 4;
        le[0] += a <= 1;
        le[1] += a <= 2;
        le[2] += a <= 4;
        le[3] += a <= 8;
    }
    qsort(s, 16, sizeof(int), cmp_int);
    for (int i = 0; i < 16; i++) {
        f[i] = s[i] / 32.0;
        f[16 + i] = r[i] / 32.0;
    }
    const double mean = sum / 16.0;
    double var = sum2 / 16.0 - mean * mean;
    if (var < 0.0)
        var = 0.0;
    f[32] = mean / 32.0;
    f[33] = sqrt(var) / 32.0;
    f[34] = mn / 32.0;
    f[35] = mx / 32.0;
    f[36] = (mx - mn) / 64.0;
    f[37] = amax / 32.0;
    f[38] = l1 / 256.0;
    f[39] = nz / 16.0;
    f[40] = odd / 16.0;
    f[41] = m4 / 16.0;
    f[42] = m8 / 16.0;
    for (int i = 0; i < 4; i++)
        f[43 + i] = le[i] / 16.0;
    f[47] = log2((double)(mx - mn) + 1.0) / 10.0;
}

/*
 * Oracle: bounded integer sequence encoding -- TEST INFRASTRUCTURE ONLY.
 *
 * Section 3.3: SRV blocks are stored with BISE, the ASTC packing of integers
 * in [0, N) where N is 2^b (plain bits), 3*2^b (one trit per value plus b
 * bits) or 5*2^b (one quint per value plus b bits).  Trits are packed five to
 * an 8-bit word (3^5 = 243 < 256) and quints three to a 7-bit word
 * (5^3 = 125 < 128), which gives the closed-form lengths
 *     bits   : n*b
 *     trits  : n*b + ceil(8n/5)
 *     quints : n*b + ceil(7n/3).
 * The paper does not print a bit layout; the reading used here (stream
 * format v1) is: digit words first, group g of a trit block at bit 8g
 * (quint: 7g), a short last group of j values taking ceil(8j/5) (ceil(7j/3))
 * bits, then the n low-bit fields m_v at D + v*b, D = the digit bits.
 * Digits inside a word are base 3 (base 5), value e of the group the e-th
 * digit.  Bit p of a byte buffer is bit (p mod 8) of byte floor(p/8).
 */
#include "oracle.h"

static int g_modeN[OR_NMODES], g_modeKind[OR_NMODES], g_modeB[OR_NMODES];

/* The 28 ranges {2^b, b<=10} u {3*2^b, b<=8} u {5*2^b, b<=7}, sorted by N.
   Built once when the library is loaded. */
__attribute__((constructor)) static void build_mode_table(void)
{
    int n = 0;
    for (int b = 0; b <= 10; b++) {
        g_modeN[n] = 1 << b; g_modeKind[n] = 0; g_modeB[n] = b; n++;
    }
    for (int b = 0; b <= 8; b++) {
        g_modeN[n] = 3 << b; g_modeKind[n] = 1; g_modeB[n] = b; n++;
    }
    for (int b = 0; b <= 7; b++) {
        g_modeN[n] = 5 << b; g_modeKind[n] = 2; g_modeB[n] = b; n++;
    }
    /* selection sort by N (all N are distinct) */
    for (int i = 0; i < n; i++) {
        int best = i;
        for (int j = i + 1; j < n; j++)
            if (g_modeN[j] < g_modeN[best])
                best = j;
        int tN = g_modeN[i], tK = g_modeKind[i], tB = g_modeB[i];
        g_modeN[i] = g_modeN[best]; g_modeKind[i] = g_modeKind[best]; g_modeB[i] = g_modeB[best];
        g_modeN[best] = tN; g_modeKind[best] = tK; g_modeB[best] = tB;
    }
}

int or_mode_N(int k) { return (k >= 0 && k < OR_NMODES) ? g_modeN[k] : -1; }
int or_mode_kind(int k) { return (k >= 0 && k < OR_NMODES) ? g_modeKind[k] : -1; }
int or_mode_b(int k) { return (k >= 0 && k < OR_NMODES) ? g_modeB[k] : -1; }

static long ceil_div(long a, long b) { return (a + b - 1) / b; }

static long digit_bits(int kind, int n)
{
    if (kind == 1)
        return ceil_div(8L * n, 5);
    if (kind == 2)
        return ceil_div(7L * n, 3);
    return 0;
}

long or_bise_bits(int n, int k)
{
    if (k < 0 || k >= OR_NMODES || n < 0)
        return -1;
    return (long)n * g_modeB[k] + digit_bits(g_modeKind[k], n);
}

/* Exhaustive search over the mode table: the cheapest mode whose range holds
   every value 0..span; ties go to the smaller mode index. */
int or_choose_mode_search(int n, int span)
{
    int best = -1;
    long best_cost = 0;
    for (int k = 0; k < OR_NMODES; k++) {
        if (g_modeN[k] < span + 1)
            continue;
        long cost = or_bise_bits(n, k);
        if (best < 0 || cost < best_cost) {
            best = k;
            best_cost = cost;
        }
    }
    return best;
}

void or_put_bits(uint8_t *buf, long pos, int width, uint32_t value)
{
    for (int e = 0; e < width; e++) {
        if ((value >> e) & 1u) {
            long p = pos + e;
            buf[p >> 3] |= (uint8_t)(1u << (p & 7));
        }
    }
}

uint32_t or_get_bits(const uint8_t *buf, long pos, int width)
{
    uint32_t v = 0;
    for (int e = 0; e < width; e++) {
        long p = pos + e;
        v |= (uint32_t)((buf[p >> 3] >> (p & 7)) & 1u) << e;
    }
    return v;
}

static int group_size(int kind) { return kind == 1 ? 5 : 3; }
static int digit_base(int kind) { return kind == 1 ? 3 : 5; }
static int full_word_bits(int kind) { return kind == 1 ? 8 : 7; }

void or_bise_pack(uint8_t *buf, long pos, int n, int k, const int *u)
{
    int kind = g_modeKind[k], b = g_modeB[k];
    long D = digit_bits(kind, n);
    if (kind != 0) {
        int gs = group_size(kind), base = digit_base(kind);
        int ngroups = (n + gs - 1) / gs;
        for (int g = 0; g < ngroups; g++) {
            int j = n - g * gs;
            if (j > gs)
                j = gs;
            uint32_t word = 0, scale = 1;
            for (int e = 0; e < j; e++) {
                uint32_t digit = (uint32_t)u[g * gs + e] >> b;
                word += digit * scale;
                scale *= (uint32_t)base;
            }
            or_put_bits(buf, pos + (long)g * full_word_bits(kind), (int)digit_bits(kind, j), word);
        }
    }
    for (int v = 0; v < n; v++) {
        uint32_t low = (uint32_t)u[v] & ((1u << b) - 1u);
        or_put_bits(buf, pos + D + (long)v * b, b, low);
    }
}

void or_bise_unpack(const uint8_t *buf, long pos, int n, int k, int *u)
{
    int kind = g_modeKind[k], b = g_modeB[k];
    long D = digit_bits(kind, n);
    for (int v = 0; v < n; v++)
        u[v] = (int)or_get_bits(buf, pos + D + (long)v * b, b);
    if (kind != 0) {
        int gs = group_size(kind), base = digit_base(kind);
        int ngroups = (n + gs - 1) / gs;
        for (int g = 0; g < ngroups; g++) {
            int j = n - g * gs;
            if (j > gs)
                j = gs;
            uint32_t word = or_get_bits(buf, pos + (long)g * full_word_bits(kind),
                                        (int)digit_bits(kind, j));
            for (int e = 0; e < j; e++) {
                int digit = (int)(word % (uint32_t)base);
                word /= (uint32_t)base;
                u[g * gs + e] += digit << b;
            }
        }
    }
}

/* Brute force over every sequence in [0, N_k)^n (when there are at most
   max_count of them): pack at an odd bit offset, unpack, compare, and check
   that no bit outside [pos, pos + or_bise_bits) was set.  Returns the number
   of failing sequences, or -1 when the enumeration is larger than max_count. */
long or_bise_exhaustive(int n, int k, long max_count)
{
    long N = g_modeN[k], count = 1;
    for (int i = 0; i < n; i++) {
        count *= N;
        if (count > max_count)
            return -1;
    }
    const long pos = 3;
    long bits = or_bise_bits(n, k);
    long nbytes = (pos + bits + 7) / 8 + 8;
    uint8_t buf[256];
    int u[64], back[64];
    long failures = 0;
    for (long idx = 0; idx < count; idx++) {
        long rest = idx;
        for (int i = 0; i < n; i++) {
            u[i] = (int)(rest % N);
            rest /= N;
        }
        for (long b = 0; b < nbytes; b++)
            buf[b] = 0;
        or_bise_pack(buf, pos, n, k, u);
        or_bise_unpack(buf, pos, n, k, back);
        int bad = 0;
        for (int i = 0; i < n; i++)
            if (back[i] != u[i])
                bad = 1;
        for (long p = 0; p < 8 * nbytes; p++)
            if ((p < pos || p >= pos + bits) && or_get_bits(buf, p, 1))
                bad = 1;
        failures += bad;
    }
    return failures;
}

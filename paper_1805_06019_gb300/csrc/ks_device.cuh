// Device functions of the learned encoder aid's per-block (shift, mode)
// choice, shared by the encoder and the standalone search.  Included inside
// the including file's namespace, after its constant tables c_rangeN (the 28
// ranges, ascending) and c_modes (RLFC_MODE_TABLE_INIT).
#pragma once

// (shift, mode) candidate test and cost of the learned aid's mode space:
// qv = sign(r) floor((|r| + h) / 2^(q+s)); a candidate's range holds the span
// of qv, its minimum fits the header, and a shift s > 0 adds at most tau_err;
// cost = 256 * payload bits + lam_q8 * SSE.
__device__ __forceinline__ bool ks_cost(const int r[kVals], uint32_t q, uint32_t s, uint32_t k, int32_t tau_err,
                                        uint32_t lam_q8, long long &cost)
{
    const uint32_t t = q + s;
    const int h = t > 0 ? 1 << (t - 1) : 0;
    int mn = 0, mx = 0, maxerr = 0;
    long long sse = 0;
#pragma unroll
    for (int i = 0; i < kVals; i++) {
        const int m = (abs(r[i]) + h) >> t;
        const int qv = r[i] < 0 ? -m : m;
        mn = i == 0 ? qv : min(mn, qv);
        mx = i == 0 ? qv : max(mx, qv);
        const int e = abs(r[i] - qv * (1 << t));
        maxerr = max(maxerr, e);
        sse += (long long)e * e;
    }
    if (k >= (uint32_t)kNumModes || (int)c_rangeN[k] < mx - mn + 1 || mn < -1024 || mn > 1023)
        return false;
    if (s > 0 && maxerr > tau_err)
        return false;
    cost = 256ll * mode_bits(c_modes[k]) + (long long)lam_q8 * sse;
    return true;
}

// Exhaustive (shift, mode) search: for each shift only the smallest range
// that holds the span can win (payload lengths grow strictly with the
// range), so the 112 pairs reduce to four candidates; the first pair of least
// cost in (s, k) order wins.
__device__ __forceinline__ bool ks_search(const int r[kVals], uint32_t q, int32_t tau_err, uint32_t lam_q8,
                                          uint32_t &k_out, uint32_t &s_out)
{
    bool found = false;
    long long best = 0;
    for (uint32_t s = 0; s < 4; s++) {
        const uint32_t t = q + s;
        const int h = t > 0 ? 1 << (t - 1) : 0;
        int mn = 0, mx = 0;
#pragma unroll
        for (int i = 0; i < kVals; i++) {
            const int m = (abs(r[i]) + h) >> t;
            const int qv = r[i] < 0 ? -m : m;
            mn = i == 0 ? qv : min(mn, qv);
            mx = i == 0 ? qv : max(mx, qv);
        }
        if (mx - mn > 1023)
            continue;
        uint32_t k = 0;
        while (k < kNumModes - 1 && (int)c_rangeN[k] < mx - mn + 1)
            k++;
        long long c;
        if (ks_cost(r, q, s, k, tau_err, lam_q8, c) && (!found || c < best)) {
            best = c;
            k_out = k;
            s_out = s;
            found = true;
        }
    }
    return found;
}

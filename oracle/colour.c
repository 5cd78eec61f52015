/*
 * Oracle: lossless YCoCg-R colour transform -- TEST INFRASTRUCTURE ONLY.
 *
 * Section 4 of the paper decorrelates RGB with the lossless YCoCg-R lifting
 * transform of Malvar & Sullivan and keeps every later stage in integers.
 * ">>" below is the arithmetic (flooring) shift; the helper makes that explicit
 * so the result does not depend on how the compiler treats negative shifts.
 */
#include "oracle.h"

static int floor_half(int x)
{
    /* floor(x / 2) for any sign */
    if (x >= 0)
        return x / 2;
    return -((-x + 1) / 2);
}

/* forward lifting: Co = R - B, t = B + Co/2, Cg = G - t, Y = t + Cg/2 */
void or_ycocg_fwd(int r, int g, int b, int *y, int *co, int *cg)
{
    int c_o = r - b;
    int t = b + floor_half(c_o);
    int c_g = g - t;
    *y = t + floor_half(c_g);
    *co = c_o;
    *cg = c_g;
}

/* inverse lifting, the forward steps undone in reverse order */
void or_ycocg_inv(int y, int co, int cg, int *r, int *g, int *b)
{
    int t = y - floor_half(cg);
    int gg = cg + t;
    int bb = t - floor_half(co);
    *r = bb + co;
    *g = gg;
    *b = bb;
}

void or_ycocg_fwd_array(const uint8_t *rgb, long npx, int32_t *out)
{
    for (long i = 0; i < npx; i++) {
        int y, co, cg;
        or_ycocg_fwd(rgb[3 * i], rgb[3 * i + 1], rgb[3 * i + 2], &y, &co, &cg);
        out[3 * i] = y;
        out[3 * i + 1] = co;
        out[3 * i + 2] = cg;
    }
}

void or_ycocg_inv_array(const int32_t *ycc, long npx, int32_t *out)
{
    for (long i = 0; i < npx; i++) {
        int r, g, b;
        or_ycocg_inv(ycc[3 * i], ycc[3 * i + 1], ycc[3 * i + 2], &r, &g, &b);
        out[3 * i] = r;
        out[3 * i + 1] = g;
        out[3 * i + 2] = b;
    }
}

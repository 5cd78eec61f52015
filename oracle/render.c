/*
 * Oracle: new-view rendering, Section 3.6 -- TEST INFRASTRUCTURE ONLY.
 *
 * A ray (u, v, s, t) of a new view is interpolated quadrilinearly from 16
 * decoded samples: bilinear over the 2 x 2 nearest views on the camera plane
 * and, in each of those views, bilinear over the 2 x 2 nearest pixels.  The
 * paper does not fix the ray geometry; the reading (the dynamically
 * reparameterised focal plane of Isaksen et al., which the paper cites for
 * its renderer) is:
 *   - the new camera sits at continuous grid coordinates (u, v) in
 *     [0, U-1] x [0, V-1], views one unit apart;
 *   - the focal plane has disparity d pixels per unit of camera motion;
 *   - output pixel (x, y) of an out_w x out_h image looks along
 *     s = (x + 0.5) W / out_w - 0.5, t = (y + 0.5) H / out_h - 0.5;
 *   - in view (i, j) that ray lands at (s + d (i - u), t + d (j - v));
 *   - neighbours i0 = min(floor(u), U-2), i1 = i0 + 1, weights 1-fu, fu
 *     (one view only when U = 1), the same for v;
 *   - pixel neighbours clamp to the image edge.
 * Values are the decoded RGB divided by 255.  Arithmetic is double precision.
 */
#include <math.h>

#include "oracle.h"

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

static void axis_neighbours(double u, int G, int *i0, int *i1, double *f)
{
    if (u < 0.0)
        u = 0.0;
    if (u > G - 1)
        u = G - 1;
    if (G == 1) {
        *i0 = 0;
        *i1 = 0;
        *f = 0.0;
        return;
    }
    int a = (int)floor(u);
    if (a > G - 2)
        a = G - 2;
    *i0 = a;
    *i1 = a + 1;
    *f = u - a;
}

/* bilinear sample of one decoded view at continuous pixel (xs, ys) */
static void sample_view(const uint8_t *img, int W, int H, double xs, double ys, double *rgb)
{
    int x0 = (int)floor(xs), y0 = (int)floor(ys);
    double fx = xs - x0, fy = ys - y0;
    int xa = clampi(x0, 0, W - 1), xb = clampi(x0 + 1, 0, W - 1);
    int ya = clampi(y0, 0, H - 1), yb = clampi(y0 + 1, 0, H - 1);
    for (int c = 0; c < 3; c++) {
        double p00 = img[((long)ya * W + xa) * 3 + c];
        double p10 = img[((long)ya * W + xb) * 3 + c];
        double p01 = img[((long)yb * W + xa) * 3 + c];
        double p11 = img[((long)yb * W + xb) * 3 + c];
        double top = (1.0 - fx) * p00 + fx * p10;
        double bot = (1.0 - fx) * p01 + fx * p11;
        rgb[c] = ((1.0 - fy) * top + fy * bot) / 255.0;
    }
}

void or_render_pixel(const uint8_t *lf, int U, int V, int W, int H,
                     double u, double v, double d, int out_w, int out_h,
                     int x, int y, double *out)
{
    int i0, i1, j0, j1;
    double fu, fv;
    /* the camera stays on the grid */
    u = u < 0.0 ? 0.0 : (u > U - 1 ? U - 1 : u);
    v = v < 0.0 ? 0.0 : (v > V - 1 ? V - 1 : v);
    axis_neighbours(u, U, &i0, &i1, &fu);
    axis_neighbours(v, V, &j0, &j1, &fv);
    double s = (x + 0.5) * W / out_w - 0.5;
    double t = (y + 0.5) * H / out_h - 0.5;
    int iv[2] = {i0, i1}, jv[2] = {j0, j1};
    double wu[2] = {1.0 - fu, fu}, wv[2] = {1.0 - fv, fv};
    out[0] = out[1] = out[2] = 0.0;
    for (int b = 0; b < 2; b++) {
        for (int a = 0; a < 2; a++) {
            double w = wu[a] * wv[b];
            if (w == 0.0)
                continue;
            int i = iv[a], j = jv[b];
            const uint8_t *img = lf + ((long)j * U + i) * W * H * 3;
            double rgb[3];
            sample_view(img, W, H, s + d * (i - u), t + d * (j - v), rgb);
            for (int c = 0; c < 3; c++)
                out[c] += w * rgb[c];
        }
    }
}

void or_render_view(const uint8_t *lf, int U, int V, int W, int H,
                    double u, double v, double d, int out_w, int out_h, double *out)
{
    for (int y = 0; y < out_h; y++)
        for (int x = 0; x < out_w; x++)
            or_render_pixel(lf, U, V, W, H, u, v, d, out_w, out_h, x, y,
                            out + ((long)y * out_w + x) * 3);
}

/*
 * Oracle: the learned encoder aid's network in FP64 -- TEST INFRASTRUCTURE
 * ONLY.
 *
 * A multilayer perceptron from the 48 block statistics of or_ks_features to
 * a softmax over the 112 (shift, mode) classes of the block header (class
 * s * 28 + k): 48 -> 64 (ReLU) -> 64 (ReLU) -> 112.  Parameters, flat and in
 * this order:
 *   W1 [64][48], b1 [64], W2 [64][64], b2 [64], W3 [112][64], b3 [112]
 * (rows are output units).  The loss of a sample is the cross-entropy
 * -log softmax(z)[y]; losses and gradients are summed over the samples.
 * The backward pass is the chain rule written out layer by layer; the
 * derivative of the ReLU is taken as 1 where its output is positive.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

#define NI 48
#define NH 64
#define NO 112

static const double *W1(const double *w) { return w; }
static const double *B1(const double *w) { return w + NH * NI; }
static const double *W2(const double *w) { return w + NH * NI + NH; }
static const double *B2(const double *w) { return w + NH * NI + NH + NH * NH; }
static const double *W3(const double *w) { return w + NH * NI + NH + NH * NH + NH; }
static const double *B3(const double *w) { return w + NH * NI + NH + NH * NH + NH + NO * NH; }

int or_mlp_nparams(void) { return NH * NI + NH + NH * NH + NH + NO * NH + NO; }

static void forward_one(const double *w, const double *x, double *h1, double *h2, double *z)
{
    for (int j = 0; j < NH; j++) {
        double a = B1(w)[j];
        for (int i = 0; i < NI; i++)
            a += W1(w)[j * NI + i] * x[i];
        h1[j] = a > 0.0 ? a : 0.0;
    }
    for (int j = 0; j < NH; j++) {
        double a = B2(w)[j];
        for (int i = 0; i < NH; i++)
            a += W2(w)[j * NH + i] * h1[i];
        h2[j] = a > 0.0 ? a : 0.0;
    }
    for (int j = 0; j < NO; j++) {
        double a = B3(w)[j];
        for (int i = 0; i < NH; i++)
            a += W3(w)[j * NH + i] * h2[i];
        z[j] = a;
    }
}

void or_mlp_forward(const double *w, const double *x, int n, double *logits)
{
    double h1[NH], h2[NH];
    for (int s = 0; s < n; s++)
        forward_one(w, x + (long)s * NI, h1, h2, logits + (long)s * NO);
}

int or_mlp_loss_grad(const double *w, const double *x, const int *y, int n, double *grad, double *loss)
{
    const int P = or_mlp_nparams();
    memset(grad, 0, sizeof(double) * P);
    double *gW1 = grad, *gB1 = grad + NH * NI, *gW2 = gB1 + NH, *gB2 = gW2 + NH * NH, *gW3 = gB2 + NH,
           *gB3 = gW3 + NO * NH;
    double h1[NH], h2[NH], z[NO], dz[NO], dh2[NH], dh1[NH];
    double total = 0.0;
    for (int s = 0; s < n; s++) {
        const double *xs = x + (long)s * NI;
        if (y[s] < 0 || y[s] >= NO)
            return -1;
        forward_one(w, xs, h1, h2, z);
        double zmax = z[0];
        for (int j = 1; j < NO; j++)
            if (z[j] > zmax) zmax = z[j];
        double den = 0.0;
        for (int j = 0; j < NO; j++)
            den += exp(z[j] - zmax);
        total += -(z[y[s]] - zmax - log(den));
        /* d loss / d z = softmax(z) - onehot(y) */
        for (int j = 0; j < NO; j++)
            dz[j] = exp(z[j] - zmax) / den - (j == y[s] ? 1.0 : 0.0);
        for (int j = 0; j < NO; j++) {
            gB3[j] += dz[j];
            for (int i = 0; i < NH; i++)
                gW3[j * NH + i] += dz[j] * h2[i];
        }
        for (int i = 0; i < NH; i++) {
            double a = 0.0;
            for (int j = 0; j < NO; j++)
                a += W3(w)[j * NH + i] * dz[j];
            dh2[i] = h2[i] > 0.0 ? a : 0.0;
        }
        for (int j = 0; j < NH; j++) {
            gB2[j] += dh2[j];
            for (int i = 0; i < NH; i++)
                gW2[j * NH + i] += dh2[j] * h1[i];
        }
        for (int i = 0; i < NH; i++) {
            double a = 0.0;
            for (int j = 0; j < NH; j++)
                a += W2(w)[j * NH + i] * dh2[j];
            dh1[i] = h1[i] > 0.0 ? a : 0.0;
        }
        for (int j = 0; j < NH; j++) {
            gB1[j] += dh1[j];
            for (int i = 0; i < NI; i++)
                gW1[j * NI + i] += dh1[j] * xs[i];
        }
    }
    *loss = total;
    return 0;
}

/*
 * mlp.c -- TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * FP64 reference of the temperature-guess network used by the EOS inversion:
 * y = W3 tanh(W2 tanh(W1 x + b1) + b2) + b3, with nin inputs, two hidden
 * layers of nh units and one output.  Flat weight layout:
 *   W1[nh][nin], b1[nh], W2[nh][nh], b2[nh], W3[nh], b3[1].
 * ora_mlp_loss_grad returns the mean squared error over n samples and its
 * gradient with respect to every weight (plain backpropagation: the chain rule
 * applied layer by layer, no fusion).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

static void offsets(int nin, int nh, long *o) {
  o[0] = 0;                     /* W1 */
  o[1] = o[0] + (long)nh * nin; /* b1 */
  o[2] = o[1] + nh;             /* W2 */
  o[3] = o[2] + (long)nh * nh;  /* b2 */
  o[4] = o[3] + nh;             /* W3 */
  o[5] = o[4] + nh;             /* b3 */
  o[6] = o[5] + 1;              /* total */
}

void ora_mlp_forward(const double *w, int nin, int nh, const double *x, long n, double *y) {
  long o[7];
  offsets(nin, nh, o);
  double *h1 = malloc(sizeof(double) * nh), *h2 = malloc(sizeof(double) * nh);
  for (long s = 0; s < n; ++s) {
    const double *xs = x + s * nin;
    for (int a = 0; a < nh; ++a) {
      double z = w[o[1] + a];
      for (int b = 0; b < nin; ++b) z += w[o[0] + (long)a * nin + b] * xs[b];
      h1[a] = tanh(z);
    }
    for (int a = 0; a < nh; ++a) {
      double z = w[o[3] + a];
      for (int b = 0; b < nh; ++b) z += w[o[2] + (long)a * nh + b] * h1[b];
      h2[a] = tanh(z);
    }
    double z = w[o[5]];
    for (int b = 0; b < nh; ++b) z += w[o[4] + b] * h2[b];
    y[s] = z;
  }
  free(h1); free(h2);
}

double ora_mlp_loss_grad(const double *w, int nin, int nh, const double *x,
                         const double *t, long n, double *grad) {
  long o[7];
  offsets(nin, nh, o);
  memset(grad, 0, sizeof(double) * o[6]);
  double *h1 = malloc(sizeof(double) * nh), *h2 = malloc(sizeof(double) * nh);
  double *d1 = malloc(sizeof(double) * nh), *d2 = malloc(sizeof(double) * nh);
  double loss = 0.0;
  for (long s = 0; s < n; ++s) {
    const double *xs = x + s * nin;
    for (int a = 0; a < nh; ++a) {
      double z = w[o[1] + a];
      for (int b = 0; b < nin; ++b) z += w[o[0] + (long)a * nin + b] * xs[b];
      h1[a] = tanh(z);
    }
    for (int a = 0; a < nh; ++a) {
      double z = w[o[3] + a];
      for (int b = 0; b < nh; ++b) z += w[o[2] + (long)a * nh + b] * h1[b];
      h2[a] = tanh(z);
    }
    double y = w[o[5]];
    for (int b = 0; b < nh; ++b) y += w[o[4] + b] * h2[b];
    double r = y - t[s];
    loss += r * r;
    double dy = 2.0 * r / (double)n;            /* dL/dy */
    grad[o[5]] += dy;
    for (int b = 0; b < nh; ++b) {
      grad[o[4] + b] += dy * h2[b];
      d2[b] = dy * w[o[4] + b] * (1.0 - h2[b] * h2[b]);  /* dL/dz2 */
    }
    for (int a = 0; a < nh; ++a) {
      grad[o[3] + a] += d2[a];
      for (int b = 0; b < nh; ++b) grad[o[2] + (long)a * nh + b] += d2[a] * h1[b];
    }
    for (int b = 0; b < nh; ++b) {
      double s2 = 0.0;
      for (int a = 0; a < nh; ++a) s2 += w[o[2] + (long)a * nh + b] * d2[a];
      d1[b] = s2 * (1.0 - h1[b] * h1[b]);        /* dL/dz1 */
    }
    for (int a = 0; a < nh; ++a) {
      grad[o[1] + a] += d1[a];
      for (int b = 0; b < nin; ++b) grad[o[0] + (long)a * nin + b] += d1[a] * xs[b];
    }
  }
  free(h1); free(h2); free(d1); free(d2);
  return loss / (double)n;
}

/* mlp.c -- plain FP64 restatement of the learned warm start that precedes the Krylov solve of the
 * mixed-precision frequency sweep: feature map, 4-layer perceptron, squared-error loss with its
 * analytic gradient, and one Adam step.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).  The learned warm start is not part of the paper's
 * method: the paper solves every frequency directly (Sec. 4).  Its definition lives in the
 * oracle header, written out in full, and this file follows it loop by loop:
 *
 *   features phi in R^64 of a node (x, nu) at wavenumber k, with centre c, length scale s,
 *   incidence direction d and top wavenumber kmax:
 *     phi[0..2] = (x - c)/s,  phi[3..5] = nu,  phi[6] = k/kmax,  phi[7] = (k/kmax)^2,
 *     phi[8 + 2(4j+q)] = cos(theta_jq),  phi[9 + 2(4j+q)] = sin(theta_jq),
 *     theta_jq = k * sc_q * (b_j . (x - c)),  sc = {0.5, 1, 1.5, 2},
 *     b = {d, e_x, e_y, e_z, (e_x+e_y)/sqrt2, (e_y+e_z)/sqrt2, (e_z+e_x)/sqrt2}.
 *   network: h1 = tanh(W1 phi + b1), h2 = tanh(W2 h1 + b2), h3 = tanh(W3 h2 + b3),
 *            y = W4 h3 + b4  (W1 256x64, W2 W3 256x256, W4 2x256; row-major, out x in).
 *   parameter vector theta: W1 | b1 | W2 | b2 | W3 | b3 | W4 | b4  (148 738 values).
 *   loss over a batch of B rows: L = (1/B) sum_rows sum_o (y_o - t_o)^2.
 *   Adam (Kingma & Ba, 2015): m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
 *     theta -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

#define D_IN 64
#define W_H 256
#define D_OUT 2

enum {
  OFF_W1 = 0,
  OFF_B1 = OFF_W1 + W_H * D_IN,
  OFF_W2 = OFF_B1 + W_H,
  OFF_B2 = OFF_W2 + W_H * W_H,
  OFF_W3 = OFF_B2 + W_H,
  OFF_B3 = OFF_W3 + W_H * W_H,
  OFF_W4 = OFF_B3 + W_H,
  OFF_B4 = OFF_W4 + D_OUT * W_H,
  N_PARAM = OFF_B4 + D_OUT
};

int64_t or_mlp_param_count(void) { return N_PARAM; }

int or_mlp_features(const double* x, const double* nu, int64_t N, const double* kv, int64_t nk,
                    const double* dir, const double* centre, double scale, double kmax, double* phi) {
  if (N < 0 || nk < 0 || !(scale > 0) || !(kmax > 0)) return -1;
  const double r2 = sqrt(0.5);
  const double b[7][3] = {{dir[0], dir[1], dir[2]}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1},
                          {r2, r2, 0}, {0, r2, r2}, {r2, 0, r2}};
  const double sc[4] = {0.5, 1.0, 1.5, 2.0};
  for (int64_t m = 0; m < nk; ++m) {
    const double k = kv[m];
    for (int64_t i = 0; i < N; ++i) {
      double* f = phi + (m * N + i) * D_IN;
      double r[3];
      for (int a = 0; a < 3; ++a) r[a] = x[3 * i + a] - centre[a];
      for (int a = 0; a < 3; ++a) f[a] = r[a] / scale;
      for (int a = 0; a < 3; ++a) f[3 + a] = nu[3 * i + a];
      f[6] = k / kmax;
      f[7] = (k / kmax) * (k / kmax);
      for (int j = 0; j < 7; ++j) {
        const double proj = b[j][0] * r[0] + b[j][1] * r[1] + b[j][2] * r[2];
        for (int q = 0; q < 4; ++q) {
          const double th = k * sc[q] * proj;
          f[8 + 2 * (4 * j + q)] = cos(th);
          f[9 + 2 * (4 * j + q)] = sin(th);
        }
      }
    }
  }
  return 0;
}

/* out[o] = sum_i W[o][i] in[i] + bias[o] */
static void affine(const double* W, const double* bias, int n_out, int n_in, const double* in, double* out) {
  for (int o = 0; o < n_out; ++o) {
    double s = bias[o];
    for (int i = 0; i < n_in; ++i) s += W[o * n_in + i] * in[i];
    out[o] = s;
  }
}

/* one row forward; keeps the hidden activations for the backward pass */
static void forward_row(const double* th, const double* phi, double* h1, double* h2, double* h3, double* y) {
  affine(th + OFF_W1, th + OFF_B1, W_H, D_IN, phi, h1);
  for (int o = 0; o < W_H; ++o) h1[o] = tanh(h1[o]);
  affine(th + OFF_W2, th + OFF_B2, W_H, W_H, h1, h2);
  for (int o = 0; o < W_H; ++o) h2[o] = tanh(h2[o]);
  affine(th + OFF_W3, th + OFF_B3, W_H, W_H, h2, h3);
  for (int o = 0; o < W_H; ++o) h3[o] = tanh(h3[o]);
  affine(th + OFF_W4, th + OFF_B4, D_OUT, W_H, h3, y);
}

int or_mlp_forward(const double* theta, const double* X, int64_t B, double* Y) {
  if (B < 0) return -1;
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < B; ++r) {
    double h1[W_H], h2[W_H], h3[W_H];
    forward_row(theta, X + r * D_IN, h1, h2, h3, Y + r * D_OUT);
  }
  return 0;
}

/* Backward by the chain rule, layer by layer from the output:
 *   dy = 2 (y - t) / B;  dW4 += dy h3^T, db4 += dy;  dh3 = W4^T dy;  dz3 = dh3 (1 - h3^2);
 *   dW3 += dz3 h2^T, db3 += dz3;  dh2 = W3^T dz3;  dz2 = dh2 (1 - h2^2);  ... down to dW1 += dz1 phi^T. */
int or_mlp_loss_grad(const double* theta, const double* X, const double* T, int64_t B, double* loss,
                     double* grad) {
  if (B <= 0) return -1;
  memset(grad, 0, sizeof(double) * N_PARAM);
  double L = 0.0;
#pragma omp parallel
  {
    double* g = (double*)calloc(N_PARAM, sizeof(double));
    double Lp = 0.0;
#pragma omp for schedule(static)
    for (int64_t r = 0; r < B; ++r) {
      double h1[W_H], h2[W_H], h3[W_H], y[D_OUT], dy[D_OUT];
      double dz3[W_H], dz2[W_H], dz1[W_H];
      const double* phi = X + r * D_IN;
      forward_row(theta, phi, h1, h2, h3, y);
      for (int o = 0; o < D_OUT; ++o) {
        const double e = y[o] - T[r * D_OUT + o];
        Lp += e * e / (double)B;
        dy[o] = 2.0 * e / (double)B;
      }
      for (int o = 0; o < D_OUT; ++o) {
        for (int i = 0; i < W_H; ++i) g[OFF_W4 + o * W_H + i] += dy[o] * h3[i];
        g[OFF_B4 + o] += dy[o];
      }
      for (int i = 0; i < W_H; ++i) {
        double s = 0.0;
        for (int o = 0; o < D_OUT; ++o) s += theta[OFF_W4 + o * W_H + i] * dy[o];
        dz3[i] = s * (1.0 - h3[i] * h3[i]);
      }
      for (int o = 0; o < W_H; ++o) {
        for (int i = 0; i < W_H; ++i) g[OFF_W3 + o * W_H + i] += dz3[o] * h2[i];
        g[OFF_B3 + o] += dz3[o];
      }
      for (int i = 0; i < W_H; ++i) {
        double s = 0.0;
        for (int o = 0; o < W_H; ++o) s += theta[OFF_W3 + o * W_H + i] * dz3[o];
        dz2[i] = s * (1.0 - h2[i] * h2[i]);
      }
      for (int o = 0; o < W_H; ++o) {
        for (int i = 0; i < W_H; ++i) g[OFF_W2 + o * W_H + i] += dz2[o] * h1[i];
        g[OFF_B2 + o] += dz2[o];
      }
      for (int i = 0; i < W_H; ++i) {
        double s = 0.0;
        for (int o = 0; o < W_H; ++o) s += theta[OFF_W2 + o * W_H + i] * dz2[o];
        dz1[i] = s * (1.0 - h1[i] * h1[i]);
      }
      for (int o = 0; o < W_H; ++o) {
        for (int i = 0; i < D_IN; ++i) g[OFF_W1 + o * D_IN + i] += dz1[o] * phi[i];
        g[OFF_B1 + o] += dz1[o];
      }
    }
#pragma omp critical
    {
      for (int64_t p = 0; p < N_PARAM; ++p) grad[p] += g[p];
      L += Lp;
    }
    free(g);
  }
  *loss = L;
  return 0;
}

int or_mlp_loss(const double* theta, const double* X, const double* T, int64_t B, double* loss) {
  if (B <= 0) return -1;
  double L = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : L)
  for (int64_t r = 0; r < B; ++r) {
    double h1[W_H], h2[W_H], h3[W_H], y[D_OUT];
    forward_row(theta, X + r * D_IN, h1, h2, h3, y);
    for (int o = 0; o < D_OUT; ++o) {
      const double e = y[o] - T[r * D_OUT + o];
      L += e * e / (double)B;
    }
  }
  *loss = L;
  return 0;
}

int or_adam_step(int64_t P, double* theta, const double* grad, double* m, double* v, int64_t t, double lr,
                 double beta1, double beta2, double eps) {
  if (P < 0 || t < 1) return -1;
  const double c1 = 1.0 - pow(beta1, (double)t), c2 = 1.0 - pow(beta2, (double)t);
  for (int64_t p = 0; p < P; ++p) {
    m[p] = beta1 * m[p] + (1.0 - beta1) * grad[p];
    v[p] = beta2 * v[p] + (1.0 - beta2) * grad[p] * grad[p];
    theta[p] -= lr * (m[p] / c1) / (sqrt(v[p] / c2) + eps);
  }
  return 0;
}

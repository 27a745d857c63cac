/*
 * mlp_oracle.c -- FP64 CPU oracle of the learned stress closure: a plain MLP
 * with exact (erf) GELU, mean-squared-error loss, reverse-mode gradient and
 * one AdamW step (Loshchilov & Hutter, "Decoupled weight decay
 * regularization", ICLR 2019).  The paper has no learned closure; the
 * network exists only in this library's surrogate-gated macro step.
 *
 * TEST INFRASTRUCTURE ONLY (see lhmm_oracle.h).
 */
#include "lhmm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

double orc_gelu(double x) { return 0.5 * x * (1.0 + erf(x / sqrt(2.0))); }

static double gelu_grad(double x) {
  return 0.5 * (1.0 + erf(x / sqrt(2.0))) + x * exp(-0.5 * x * x) / sqrt(2.0 * M_PI);
}

long orc_mlp_n_params(int n_layers, const int* dims) {
  long n = 0;
  for (int l = 0; l < n_layers; ++l) n += (long)dims[l + 1] * dims[l] + dims[l + 1];
  return n;
}

/* pre-activations z_l (dims[l+1] x batch) and activations h_l (dims[l] x batch) */
static void forward_all(int n_layers, const int* dims, const double* params, int batch,
                        const double* x, double** h, double** z) {
  for (int k = 0; k < batch; ++k)
    for (int i = 0; i < dims[0]; ++i) h[0][(long)k * dims[0] + i] = x[(long)k * dims[0] + i];
  const double* w = params;
  for (int l = 0; l < n_layers; ++l) {
    const int nin = dims[l], nout = dims[l + 1];
    const double* W = w;
    const double* bias = w + (long)nout * nin;
    for (int k = 0; k < batch; ++k) {
      for (int o = 0; o < nout; ++o) {
        double s = bias[o];
        for (int i = 0; i < nin; ++i) s += W[(long)o * nin + i] * h[l][(long)k * nin + i];
        z[l][(long)k * nout + o] = s;
        h[l + 1][(long)k * nout + o] = (l < n_layers - 1) ? orc_gelu(s) : s;
      }
    }
    w += (long)nout * nin + nout;
  }
}

static void alloc_acts(int n_layers, const int* dims, int batch, double*** h, double*** z) {
  *h = (double**)malloc(sizeof(double*) * (n_layers + 1));
  *z = (double**)malloc(sizeof(double*) * n_layers);
  for (int l = 0; l <= n_layers; ++l) (*h)[l] = (double*)malloc(sizeof(double) * batch * dims[l]);
  for (int l = 0; l < n_layers; ++l) (*z)[l] = (double*)malloc(sizeof(double) * batch * dims[l + 1]);
}

static void free_acts(int n_layers, double** h, double** z) {
  for (int l = 0; l <= n_layers; ++l) free(h[l]);
  for (int l = 0; l < n_layers; ++l) free(z[l]);
  free(h);
  free(z);
}

void orc_mlp_forward(int n_layers, const int* dims, const double* params, int batch,
                     const double* x, double* y) {
  double **h, **z;
  alloc_acts(n_layers, dims, batch, &h, &z);
  forward_all(n_layers, dims, params, batch, x, h, z);
  memcpy(y, h[n_layers], sizeof(double) * batch * dims[n_layers]);
  free_acts(n_layers, h, z);
}

double orc_mlp_loss_grad(int n_layers, const int* dims, const double* params, int batch,
                         const double* x, const double* target, double* grad) {
  double **h, **z;
  alloc_acts(n_layers, dims, batch, &h, &z);
  forward_all(n_layers, dims, params, batch, x, h, z);
  const int nout = dims[n_layers];
  const double denom = (double)batch * nout;
  double loss = 0.0;
  /* delta = d loss / d z of the current layer */
  double* delta = (double*)malloc(sizeof(double) * batch * nout);
  for (long k = 0; k < (long)batch * nout; ++k) {
    double e = h[n_layers][k] - target[k];
    loss += e * e;
    delta[k] = 2.0 * e / denom;
  }
  loss /= denom;
  /* parameter offsets of each layer */
  long* off = (long*)malloc(sizeof(long) * n_layers);
  long o = 0;
  for (int l = 0; l < n_layers; ++l) { off[l] = o; o += (long)dims[l + 1] * dims[l] + dims[l + 1]; }
  for (int l = n_layers - 1; l >= 0; --l) {
    const int nin = dims[l], no = dims[l + 1];
    const double* W = params + off[l];
    double* gW = grad + off[l];
    double* gb = grad + off[l] + (long)no * nin;
    for (int oo = 0; oo < no; ++oo) {
      double sb = 0.0;
      for (int k = 0; k < batch; ++k) sb += delta[(long)k * no + oo];
      gb[oo] = sb;
      for (int i = 0; i < nin; ++i) {
        double s = 0.0;
        for (int k = 0; k < batch; ++k) s += delta[(long)k * no + oo] * h[l][(long)k * nin + i];
        gW[(long)oo * nin + i] = s;
      }
    }
    if (l > 0) {
      double* nd = (double*)malloc(sizeof(double) * batch * nin);
      for (int k = 0; k < batch; ++k) {
        for (int i = 0; i < nin; ++i) {
          double s = 0.0;
          for (int oo = 0; oo < no; ++oo) s += W[(long)oo * nin + i] * delta[(long)k * no + oo];
          nd[(long)k * nin + i] = s * gelu_grad(z[l - 1][(long)k * nin + i]);
        }
      }
      free(delta);
      delta = nd;
    }
  }
  free(delta);
  free(off);
  free_acts(n_layers, h, z);
  return loss;
}

void orc_adamw_step(long n, double* params, const double* grad, double* m, double* v, double lr,
                    double beta1, double beta2, double eps, double wd, long t) {
  double bc1 = 1.0 - pow(beta1, (double)t);
  double bc2 = 1.0 - pow(beta2, (double)t);
  for (long k = 0; k < n; ++k) {
    m[k] = beta1 * m[k] + (1.0 - beta1) * grad[k];
    v[k] = beta2 * v[k] + (1.0 - beta2) * grad[k] * grad[k];
    double mh = m[k] / bc1;
    double vh = v[k] / bc2;
    params[k] = params[k] * (1.0 - lr * wd) - lr * mh / (sqrt(vh) + eps);
  }
}

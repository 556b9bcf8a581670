// Oracle of the learned importance-sampling proposal (test infrastructure
// only; see qcams_oracle.cpp for the rules that apply to the whole oracle).
//
// The network of the learned-proposal extension (not part of the paper): 8 inputs (E_col,
// b, v, j, theta, phi, chi, eta), three hidden layers of width 64 with the
// SiLU activation z sigmoid(z), 4 outcome logits (Q, R_AC, R_BC, D), softmax
// cross-entropy loss, Adam (Kingma & Ba, "Adam: a method for stochastic
// optimization", ICLR 2015).  Everything here is plain FP64 with no
// blocking or fusion.
//
// Parameter vector layout (row-major): W1[64][8] b1[64] W2[64][64] b2[64]
// W3[64][64] b3[64] W4[4][64] b4[4]; 9,156 values.
//
// Proposal (importance sampling over the uniform measure on b^2, cos theta,
// phi, eta, chi): a grid of equal-measure cells; g_c = sqrt(eps + p_R(c)) at
// the cell centre, q_c = alpha / N + (1 - alpha) g_c / sum g; a lane drawn
// from cell c uniformly inside it carries the likelihood ratio
// w = (1 / N) / q_c, so E_q[w f] equals the uniform-measure mean of f.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

const int kIn = 8, kH = 64, kOut = 4;
const int kNP = kH * kIn + kH + kH * kH + kH + kH * kH + kH + kOut * kH + kOut;

struct View {
  const double *W1, *b1, *W2, *b2, *W3, *b3, *W4, *b4;
};
View view(const double* p) {
  View v;
  v.W1 = p; p += kH * kIn;
  v.b1 = p; p += kH;
  v.W2 = p; p += kH * kH;
  v.b2 = p; p += kH;
  v.W3 = p; p += kH * kH;
  v.b3 = p; p += kH;
  v.W4 = p; p += kOut * kH;
  v.b4 = p;
  return v;
}

double sigmoid(double z) { return 1.0 / (1.0 + std::exp(-z)); }

// z = W a + b for a layer with n_out rows and n_in columns
void affine(const double* W, const double* b, const double* a, int n_out, int n_in, double* z) {
  for (int o = 0; o < n_out; ++o) {
    double s = b[o];
    for (int i = 0; i < n_in; ++i) s += W[o * n_in + i] * a[i];
    z[o] = s;
  }
}

struct Acts {
  double x[kIn], z1[kH], a1[kH], z2[kH], a2[kH], z3[kH], a3[kH], z4[kOut];
};

void forward(const View& v, const double* x, Acts& A) {
  std::memcpy(A.x, x, sizeof(A.x));
  affine(v.W1, v.b1, A.x, kH, kIn, A.z1);
  for (int k = 0; k < kH; ++k) A.a1[k] = A.z1[k] * sigmoid(A.z1[k]);
  affine(v.W2, v.b2, A.a1, kH, kH, A.z2);
  for (int k = 0; k < kH; ++k) A.a2[k] = A.z2[k] * sigmoid(A.z2[k]);
  affine(v.W3, v.b3, A.a2, kH, kH, A.z3);
  for (int k = 0; k < kH; ++k) A.a3[k] = A.z3[k] * sigmoid(A.z3[k]);
  affine(v.W4, v.b4, A.a3, kOut, kH, A.z4);
}

// d SiLU / dz = s (1 + z (1 - s)), s = sigmoid(z)
double dsilu(double z) {
  double s = sigmoid(z);
  return s * (1.0 + z * (1.0 - s));
}

}  // namespace

extern "C" {

int oracle_mlp_num_params() { return kNP; }

// Logits for n inputs x[n][8] (already standardised).
void oracle_mlp_forward(const double* params, const double* x, int64_t n, double* logits) {
  View v = view(params);
  Acts A;
  for (int64_t s = 0; s < n; ++s) {
    forward(v, x + kIn * s, A);
    for (int k = 0; k < kOut; ++k) logits[kOut * s + k] = A.z4[k];
  }
}

// Softmax cross-entropy summed over the samples and divided by n, and its
// gradient (back propagation through the chain rule, layer by layer).
// Targets are outcome classes 0..3; a class >= 4 (AMBIG, FAIL) is skipped.
double oracle_mlp_loss_grad(const double* params, const double* x, const int32_t* label, int64_t n,
                            double* grad) {
  View v = view(params);
  std::memset(grad, 0, sizeof(double) * kNP);
  double* gW1 = grad;
  double* gb1 = gW1 + kH * kIn;
  double* gW2 = gb1 + kH;
  double* gb2 = gW2 + kH * kH;
  double* gW3 = gb2 + kH;
  double* gb3 = gW3 + kH * kH;
  double* gW4 = gb3 + kH;
  double* gb4 = gW4 + kOut * kH;
  double loss = 0.0;
  Acts A;
  for (int64_t s = 0; s < n; ++s) {
    if (label[s] < 0 || label[s] >= kOut) continue;
    forward(v, x + kIn * s, A);
    double m = A.z4[0];
    for (int k = 1; k < kOut; ++k) m = std::fmax(m, A.z4[k]);
    double sum = 0.0, p[kOut];
    for (int k = 0; k < kOut; ++k) { p[k] = std::exp(A.z4[k] - m); sum += p[k]; }
    for (int k = 0; k < kOut; ++k) p[k] /= sum;
    loss += -std::log(p[label[s]]);
    double d4[kOut], d3[kH], d2[kH], d1[kH];
    for (int k = 0; k < kOut; ++k) d4[k] = (p[k] - (k == label[s] ? 1.0 : 0.0)) / double(n);
    for (int o = 0; o < kOut; ++o) {
      gb4[o] += d4[o];
      for (int i = 0; i < kH; ++i) gW4[o * kH + i] += d4[o] * A.a3[i];
    }
    for (int i = 0; i < kH; ++i) {
      double g = 0.0;
      for (int o = 0; o < kOut; ++o) g += v.W4[o * kH + i] * d4[o];
      d3[i] = g * dsilu(A.z3[i]);
    }
    for (int o = 0; o < kH; ++o) {
      gb3[o] += d3[o];
      for (int i = 0; i < kH; ++i) gW3[o * kH + i] += d3[o] * A.a2[i];
    }
    for (int i = 0; i < kH; ++i) {
      double g = 0.0;
      for (int o = 0; o < kH; ++o) g += v.W3[o * kH + i] * d3[o];
      d2[i] = g * dsilu(A.z2[i]);
    }
    for (int o = 0; o < kH; ++o) {
      gb2[o] += d2[o];
      for (int i = 0; i < kH; ++i) gW2[o * kH + i] += d2[o] * A.a1[i];
    }
    for (int i = 0; i < kH; ++i) {
      double g = 0.0;
      for (int o = 0; o < kH; ++o) g += v.W2[o * kH + i] * d2[o];
      d1[i] = g * dsilu(A.z1[i]);
    }
    for (int o = 0; o < kH; ++o) {
      gb1[o] += d1[o];
      for (int i = 0; i < kIn; ++i) gW1[o * kIn + i] += d1[o] * A.x[i];
    }
  }
  return loss / double(n);
}

// One Adam step (bias-corrected moments), step number t >= 1.
void oracle_adam_step(double* params, double* m, double* v, const double* grad, int64_t n,
                      int64_t t, double lr, double beta1, double beta2, double eps) {
  const double c1 = 1.0 - std::pow(beta1, double(t));
  const double c2 = 1.0 - std::pow(beta2, double(t));
  for (int64_t i = 0; i < n; ++i) {
    m[i] = beta1 * m[i] + (1.0 - beta1) * grad[i];
    v[i] = beta2 * v[i] + (1.0 - beta2) * grad[i] * grad[i];
    const double mh = m[i] / c1, vh = v[i] / c2;
    params[i] -= lr * mh / (std::sqrt(vh) + eps);
  }
}

// Proposal table over a grid of cells: p_R(centre) = softmax probability of
// the two reactive classes for the features of each cell centre (x_cells,
// standardised, [n_cells][8]).  q[c] as in the header.
void oracle_proposal(const double* params, const double* x_cells, int64_t n_cells, double eps,
                     double alpha, double* q) {
  View v = view(params);
  Acts A;
  std::vector<double> g(n_cells);
  double sg = 0.0;
  for (int64_t c = 0; c < n_cells; ++c) {
    forward(v, x_cells + kIn * c, A);
    double m = A.z4[0];
    for (int k = 1; k < kOut; ++k) m = std::fmax(m, A.z4[k]);
    double e[kOut], sum = 0.0;
    for (int k = 0; k < kOut; ++k) { e[k] = std::exp(A.z4[k] - m); sum += e[k]; }
    const double pR = (e[1] + e[2]) / sum;
    g[c] = std::sqrt(eps + pR);
    sg += g[c];
  }
  for (int64_t c = 0; c < n_cells; ++c)
    q[c] = alpha / double(n_cells) + (1.0 - alpha) * g[c] / sg;
}

void oracle_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out);

// Network inputs at the centres of the proposal grid cells (equal-measure
// cells in b^2 in [0, b2_max], cos theta in [-1, 1], phi, eta in [0, 2 pi),
// chi in [0, 1)), standardised with mean / std: x[n_cells][8] = (E, b, v, j,
// theta, phi, chi, eta).
void oracle_proposal_grid(const int32_t* dims, double b2_max, double E, int32_t v, int32_t j,
                          const double* mean, const double* stdv, double* x) {
  const double pi = 3.14159265358979323846;
  int64_t c = 0;
  for (int ib = 0; ib < dims[0]; ++ib)
    for (int ic = 0; ic < dims[1]; ++ic)
      for (int ip = 0; ip < dims[2]; ++ip)
        for (int ie = 0; ie < dims[3]; ++ie)
          for (int ix = 0; ix < dims[4]; ++ix, ++c) {
            double f[8];
            f[0] = E;
            f[1] = std::sqrt(b2_max * (ib + 0.5) / dims[0]);
            f[2] = v;
            f[3] = j;
            f[4] = std::acos(2.0 * (ic + 0.5) / dims[1] - 1.0);
            f[5] = 2.0 * pi * (ip + 0.5) / dims[2];
            f[6] = (ix + 0.5) / dims[4];
            f[7] = 2.0 * pi * (ie + 0.5) / dims[3];
            for (int k = 0; k < 8; ++k) x[8 * c + k] = (f[k] - mean[k]) / stdv[k];
          }
}

// Integer form of a proposal: qfix = round(q 2^40), cdf = running sums.
void oracle_proposal_cdf(const double* q, int64_t n_cells, int64_t* qfix, int64_t* cdf) {
  int64_t run = 0;
  for (int64_t c = 0; c < n_cells; ++c) {
    qfix[c] = (int64_t)std::llrint(std::ldexp(q[c], 40));
    run += qfix[c];
    cdf[c] = run;
  }
}

// Draw n lanes from an integer proposal over the (b^2, cos theta, phi, eta,
// chi) grid dims[5]: Philox words (key seed; counters (id_lo, id_hi, 1, 0)
// and (id_lo, id_hi, 2, 0)), u = (word + 1/2) 2^-32; the cell is the first
// with cdf > floor(u_0 total); positions uniform inside it; weight
// (total / N) / qfix[cell].  Outputs b[n], u[n][4] (init uniforms), w[n],
// cell[n].
void oracle_sample_proposal(const int32_t* dims, double b2_max, const int64_t* qfix,
                            const int64_t* cdf, int64_t n_cells, int64_t n, uint64_t seed,
                            uint64_t id_offset, double* b, double* u, double* w, int32_t* cell) {
  const uint32_t key[2] = {uint32_t(seed), uint32_t(seed >> 32)};
  const unsigned __int128 total = (unsigned __int128)(uint64_t)cdf[n_cells - 1];
  for (int64_t i = 0; i < n; ++i) {
    const uint64_t id = id_offset + (uint64_t)i;
    uint32_t c1[4] = {uint32_t(id), uint32_t(id >> 32), 1u, 0u}, wa[4];
    uint32_t c2[4] = {uint32_t(id), uint32_t(id >> 32), 2u, 0u}, wb[4];
    oracle_philox4x32_10(c1, key, wa);
    oracle_philox4x32_10(c2, key, wb);
    auto uni = [](uint32_t x) { return (double(x) + 0.5) * (1.0 / 4294967296.0); };
    // floor(u_0 total) = floor((2 w + 1) total / 2^33), exactly
    const uint64_t U = (uint64_t)(((unsigned __int128)(2ull * wa[0] + 1ull) * total) >> 33);
    int64_t c = 0;
    while ((uint64_t)cdf[c] <= U) ++c;
    cell[i] = (int32_t)c;
    int64_t r = c;
    const int i_chi = (int)(r % dims[4]); r /= dims[4];
    const int i_eta = (int)(r % dims[3]); r /= dims[3];
    const int i_phi = (int)(r % dims[2]); r /= dims[2];
    const int i_cth = (int)(r % dims[1]); r /= dims[1];
    const int i_b2 = (int)r;
    b[i] = std::sqrt(b2_max * (i_b2 + uni(wa[1])) / dims[0]);
    u[4 * i + 0] = (i_cth + uni(wa[2])) / dims[1];
    u[4 * i + 1] = (i_phi + uni(wa[3])) / dims[2];
    u[4 * i + 2] = (i_eta + uni(wb[0])) / dims[3];
    u[4 * i + 3] = (i_chi + uni(wb[1])) / dims[4];
    w[i] = ((double)(uint64_t)total / (double)n_cells) / (double)qfix[c];
  }
}

// Importance-sampling estimate of the uniform-measure mean of f from lanes
// drawn from q: mean(w f) and its standard error (sample variance / n).
void oracle_is_mean(const double* w, const double* f, int64_t n, double* mean, double* se) {
  double s = 0.0, s2 = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    const double y = w[i] * f[i];
    s += y;
    s2 += y * y;
  }
  const double mu = s / double(n);
  const double var = n > 1 ? (s2 / double(n) - mu * mu) * double(n) / double(n - 1) : 0.0;
  *mean = mu;
  *se = std::sqrt(std::fmax(var, 0.0) / double(n));
}

}  // extern "C"

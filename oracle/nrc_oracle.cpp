// FP64 CPU oracle of the neural radiance cache hot path
// (Mueller, Rousselle, Novak, Keller: "Real-time Neural Radiance Caching for
// Path Tracing", ACM TOG 40(4), 2021).
//
// TEST INFRASTRUCTURE.  Only the tests, the package's smoke check and the
// benchmark's CPU-baseline and reference legs may load or call this library.
// The product path (the CUDA library) never links, imports or calls it, and
// the two share no code: every step below is written out from the paper's
// definitions, in plain loops, in double precision.  Inputs arrive as FP32
// (records, targets, weights) and are promoted to FP64.
//
// Steps and the passages they follow:
//   * training-record shuffle by a linear congruential map  - Sec. 3.5
//   * input encoding (frequency + one-blob + identity + pad) - Sec. 3.6, Table 1
//   * cheap primitives quartic / triangle wave               - Sec. 5, Fig. 7
//   * bias-free 64-wide ReLU MLP, linear RGB output          - Sec. 5 "Architecture", Fig. 4
//   * relative L2 loss, luminance normalisation              - Sec. 5, Eq. 5
//   * backward pass and weight gradients                     - Sec. 4 "Training the fully fused network"
//   * Adam                                                   - Sec. 5 "Optimizer" (Kingma & Ba 2015)
//   * exponential moving average of the weights              - Sec. 3.3, Eq. 2 (as read below)
//   * reflectance factorisation of the output                - Sec. 5 "Reflectance factorization"
//
// Readings where the paper is silent (each is listed in the design notes):
//   * the shuffle is one affine map i -> (a*i + c) mod N with gcd(a, N) = 1,
//     a and c drawn from SplitMix64(frame_seed);
//   * frequency feature d of coordinate x is sin(2^d * pi * x) (exact) or
//     tri(2^d * x - 1/2) (cheap), axis-major order;
//   * a one-blob bin holds the kernel's mass over the bin, kernel width 1/k
//     (quartic support radius 1/k; Gaussian standard deviation 1/k); no wrap;
//   * luminance = Rec. 709 weights of the stop-gradient prediction; the loss
//     is the mean over the 3*N channel terms;
//   * Adam with bias correction, eps = 1e-8 unless given, no weight decay;
//   * Eq. 2 as printed is not an average (a constant sequence does not map to
//     itself); it is read as the bias-corrected average the text describes,
//     EMA_t = ((1 - a) W_t + a eta_{t-1} EMA_{t-1}) / eta_t, eta_t = 1 - a^t;
//   * factorisation: the prediction is the network output times the sum of
//     the record's diffuse and specular albedo, channel by channel; the loss
//     compares that product with the target.
//
// Parity pins (what fixes each function other than itself) are in the tests.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <thread>
#include <vector>

namespace {

constexpr int kEncDims = 64;
constexpr int kRecFloats = 16;
constexpr int64_t kChunk = 256;  // fixed row chunk: sums do not depend on the thread count

int n_threads() {
  const char* env = std::getenv("ORACLE_THREADS");
  if (env && std::atoi(env) > 0) return std::atoi(env);
  unsigned hc = std::thread::hardware_concurrency();
  return hc ? int(hc) : 1;
}

// Runs fn(chunk_index, row_begin, row_end) over fixed chunks of kChunk rows.
template <class F>
void for_chunks(int64_t n, F fn) {
  const int64_t n_chunks = (n + kChunk - 1) / kChunk;
  const int nt = std::max(1, std::min<int>(n_threads(), int(std::max<int64_t>(n_chunks, 1))));
  if (nt == 1 || n_chunks <= 1) {
    for (int64_t c = 0; c < n_chunks; ++c) fn(c, c * kChunk, std::min(n, (c + 1) * kChunk));
    return;
  }
  std::vector<std::thread> pool;
  for (int t = 0; t < nt; ++t) {
    pool.emplace_back([=, &fn]() {
      for (int64_t c = t; c < n_chunks; c += nt) fn(c, c * kChunk, std::min(n, (c + 1) * kChunk));
    });
  }
  for (auto& th : pool) th.join();
}

uint64_t splitmix64(uint64_t& state) {
  // Steele, Lea & Flood 2014: golden-gamma increment, then the finaliser.
  state += 0x9E3779B97F4A7C15ull;
  uint64_t z = state;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

uint64_t gcd_u64(uint64_t a, uint64_t b) {
  while (b) {
    uint64_t t = a % b;
    a = b;
    b = t;
  }
  return a;
}

}  // namespace

extern "C" {

int oracle_abi_version() { return 2; }

// ---------------------------------------------------------------- Sec. 3.5 --
// The shuffle of the training records by a linear congruential generator,
// read as one affine step
// perm(i) = (a*i + c) mod N per index.  Multiplier a = 1 + 4*(h mod floor(N/4)),
// raised by 2 until coprime with N; increment c = h' mod N; (h, h') are the
// first two SplitMix64 outputs from state frame_seed.
void oracle_lcg_params(int64_t n_pool, uint64_t frame_seed, uint64_t* a_out, uint64_t* c_out) {
  const uint64_t N = uint64_t(n_pool);
  uint64_t st = frame_seed;
  const uint64_t h = splitmix64(st);
  const uint64_t h2 = splitmix64(st);
  uint64_t a = (N / 4 > 0) ? 1 + 4 * (h % (N / 4)) : 1;
  while (N > 1 && gcd_u64(a, N) != 1) a += 2;
  *a_out = a;
  *c_out = N ? h2 % N : 0;
}

void oracle_permutation(int64_t n_pool, uint64_t frame_seed, int64_t* perm) {
  uint64_t a, c;
  oracle_lcg_params(n_pool, frame_seed, &a, &c);
  const uint64_t N = uint64_t(n_pool);
  for (int64_t i = 0; i < n_pool; ++i) perm[i] = int64_t((a * uint64_t(i) + c) % N);
}

// Training batch `step` of a frame takes pool[perm(step*batch + j)], j < batch:
// the s batches of l records each are disjoint slices of one shuffle (Sec. 3.5;
// Sec. 3.3's footnote on disjoint subsets).
void oracle_gather(const float* pool, const float* target, int64_t n_pool, int64_t batch,
                   uint64_t frame_seed, int step, float* rec_out, float* tgt_out, int64_t* idx_out) {
  uint64_t a, c;
  oracle_lcg_params(n_pool, frame_seed, &a, &c);
  const uint64_t N = uint64_t(n_pool);
  for (int64_t j = 0; j < batch; ++j) {
    const uint64_t i = uint64_t(step) * uint64_t(batch) + uint64_t(j);
    const int64_t src = int64_t((a * i + c) % N);
    if (idx_out) idx_out[j] = src;
    for (int f = 0; f < kRecFloats; ++f) rec_out[j * kRecFloats + f] = pool[src * kRecFloats + f];
    for (int f = 0; f < 3; ++f) tgt_out[j * 3 + f] = target[src * 3 + f];
  }
}

// ----------------------------------------------------- Sec. 5, Fig. 7 -------
// tri(x) = 2 |x mod 2 - 1| - 1, with the floored modulo into [0, 2).
double oracle_tri(double x) {
  const double m = x - 2.0 * std::floor(x / 2.0);
  return 2.0 * std::fabs(m - 1.0) - 1.0;
}

// quartic(x) = 15/16 (1 - x^2)^2 on [-1, 1], zero outside.
double oracle_quartic(double x) {
  if (x <= -1.0 || x >= 1.0) return 0.0;
  const double t = 1.0 - x * x;
  return 15.0 / 16.0 * t * t;
}

// Antiderivative of the quartic with value 0 at 0, clamped to the support:
// Q(y) = 15/16 (y - 2 y^3 / 3 + y^5 / 5) for y in [-1, 1]; Q(+-1) = +-1/2.
double oracle_quartic_cdf(double y) {
  y = std::min(1.0, std::max(-1.0, y));
  return 15.0 / 16.0 * (y - 2.0 * y * y * y / 3.0 + y * y * y * y * y / 5.0);
}

// Frequency feature d of coordinate x (Sec. 3.6: 12 sines of frequency 2^d,
// no cosines).  enc_mode 0: the triangle wave in place of the sine (Sec. 5).
double oracle_freq_feature(double x, int d, int enc_mode) {
  const double y = std::ldexp(x, d);  // 2^d * x, exact
  if (enc_mode == 0) return oracle_tri(y - 0.5);
  return std::sin(M_PI * y);
}

// One-blob encoding of a scalar s in [0,1] into k bins [i/k, (i+1)/k): each
// bin holds the mass of a kernel of width 1/k centred at s (Mueller et al.
// 2019, cited in Sec. 3.6).  enc_mode 0: quartic kernel (Sec. 5); 1: Gaussian.
void oracle_oneblob(double s, int k, int enc_mode, double* out) {
  for (int i = 0; i < k; ++i) {
    const double lo = double(i) - k * s;  // (i/k - s) / (1/k)
    const double hi = double(i + 1) - k * s;
    if (enc_mode == 0) {
      out[i] = oracle_quartic_cdf(hi) - oracle_quartic_cdf(lo);
    } else {
      out[i] = 0.5 * (std::erf(hi / std::sqrt(2.0)) - std::erf(lo / std::sqrt(2.0)));
    }
  }
}

// Table 1 + Sec. 3.6: 36 frequency features of x, one-blob (k = 4) of
// sph(w) (8), sph(n) (8), 1 - exp(-r) (4), identity albedos (3 + 3), two pad
// entries of value pad_value (Sec. 3.6 pads with 1) -> 64 features.
void oracle_encode_one(const float* rec, int enc_mode, double pad_value, double* out) {
  int f = 0;
  for (int j = 0; j < 3; ++j)
    for (int d = 0; d < 12; ++d) out[f++] = oracle_freq_feature(double(rec[j]), d, enc_mode);
  for (int q = 3; q < 7; ++q) {  // theta_w/pi, phi_w/2pi, theta_n/pi, phi_n/2pi
    oracle_oneblob(double(rec[q]), 4, enc_mode, out + f);
    f += 4;
  }
  oracle_oneblob(-std::expm1(-double(rec[7])), 4, enc_mode, out + f);
  f += 4;
  for (int j = 8; j < 14; ++j) out[f++] = double(rec[j]);
  while (f < kEncDims) out[f++] = pad_value;
}

void oracle_encode(const float* rec, int64_t n, int enc_mode, double pad_value, double* out) {
  for_chunks(n, [&](int64_t, int64_t b, int64_t e) {
    for (int64_t r = b; r < e; ++r) oracle_encode_one(rec + r * kRecFloats, enc_mode, pad_value, out + r * kEncDims);
  });
}

// ------------------------------------------------ Sec. 5 "Architecture" -----
// n_mats bias-free layers; matrix l is dims[l+1] x dims[l], row-major
// [out][in], stored one after the other in W.  H_0 = x;
// H_{l+1} = max(0, W_l H_l) for hidden layers; the output y = W_{L-1} H_{L-1}
// is linear.  acts (optional) receives H_0 .. H_{L-1} of every row, as
// consecutive blocks acts_l[n][dims[l]].
static int64_t w_offset(const int* dims, int l) {
  int64_t off = 0;
  for (int i = 0; i < l; ++i) off += int64_t(dims[i]) * dims[i + 1];
  return off;
}

static int64_t act_offset(const int* dims, int l, int64_t n) {
  int64_t off = 0;
  for (int i = 0; i < l; ++i) off += n * dims[i];
  return off;
}

void oracle_forward(const double* W, const int* dims, int n_mats, const double* x, int64_t n, double* y,
                    double* acts) {
  int maxd = 0;
  for (int l = 0; l <= n_mats; ++l) maxd = std::max(maxd, dims[l]);
  for_chunks(n, [&](int64_t, int64_t b, int64_t e) {
    std::vector<double> h(maxd), z(maxd);
    for (int64_t r = b; r < e; ++r) {
      for (int i = 0; i < dims[0]; ++i) h[i] = x[r * dims[0] + i];
      for (int l = 0; l < n_mats; ++l) {
        if (acts) {
          double* a = acts + act_offset(dims, l, n) + r * dims[l];
          for (int i = 0; i < dims[l]; ++i) a[i] = h[i];
        }
        const double* Wl = W + w_offset(dims, l);
        for (int o = 0; o < dims[l + 1]; ++o) {
          double s = 0.0;
          for (int i = 0; i < dims[l]; ++i) s += Wl[int64_t(o) * dims[l] + i] * h[i];
          z[o] = s;
        }
        const bool last = (l == n_mats - 1);
        for (int o = 0; o < dims[l + 1]; ++o) h[o] = last ? z[o] : (z[o] > 0.0 ? z[o] : 0.0);
      }
      for (int o = 0; o < dims[n_mats]; ++o) y[r * dims[n_mats] + o] = h[o];
    }
  });
}

// --------------------------------------------------------- Sec. 5, Eq. 5 ----
// Relative L2: (y - yhat)^2 / (sg(yhat)^2 + eps).  loss_mode 0 (luminance):
// every channel is normalised by the squared luminance of the prediction
// (Rec. 709 weights); loss_mode 1: each channel by its own prediction, as
// Eq. 5 reads per scalar.  The loss is the mean over the 3*n terms; g (if not
// null) receives dL/dyhat with the denominator held constant.
double oracle_loss(const double* yhat, const float* target, int64_t n, int loss_mode, double eps, double* g) {
  const int64_t n_chunks = (n + kChunk - 1) / kChunk;
  std::vector<double> part(std::max<int64_t>(n_chunks, 1), 0.0);
  const double inv = n > 0 ? 1.0 / (3.0 * double(n)) : 0.0;
  for_chunks(n, [&](int64_t c, int64_t b, int64_t e) {
    double s = 0.0;
    for (int64_t r = b; r < e; ++r) {
      const double* p = yhat + r * 3;
      const double lum = 0.2126 * p[0] + 0.7152 * p[1] + 0.0722 * p[2];
      for (int ch = 0; ch < 3; ++ch) {
        const double norm = (loss_mode == 0 ? lum * lum : p[ch] * p[ch]) + eps;
        const double diff = p[ch] - double(target[r * 3 + ch]);
        s += diff * diff / norm;
        if (g) g[r * 3 + ch] = 2.0 * diff / norm * inv;
      }
    }
    part[c] = s;
  });
  double total = 0.0;
  for (double v : part) total += v;
  return total * inv;
}

// ------------------------------------- Sec. 4 "Training the fully fused ..." --
// delta_L = g; for l = L-1 .. 0: dW_l = sum_rows delta_{l+1} H_l^T and, for
// l >= 1, delta_l = (W_l^T delta_{l+1}) * [H_l > 0] (ReLU'(0) = 0).
// acts as written by oracle_forward.  dW has the layout of W and is
// overwritten.
void oracle_backward(const double* W, const int* dims, int n_mats, const double* acts, const double* g, int64_t n,
                     double* dW) {
  int64_t n_par = w_offset(dims, n_mats);
  int maxd = 0;
  for (int l = 0; l <= n_mats; ++l) maxd = std::max(maxd, dims[l]);
  const int64_t n_chunks = (n + kChunk - 1) / kChunk;
  std::vector<double> part(size_t(std::max<int64_t>(n_chunks, 1)) * n_par, 0.0);
  for_chunks(n, [&](int64_t c, int64_t b, int64_t e) {
    double* P = part.data() + c * n_par;
    std::vector<double> d(maxd), dn(maxd);
    for (int64_t r = b; r < e; ++r) {
      for (int o = 0; o < dims[n_mats]; ++o) d[o] = g[r * dims[n_mats] + o];
      for (int l = n_mats - 1; l >= 0; --l) {
        const double* H = acts + act_offset(dims, l, n) + r * dims[l];
        const double* Wl = W + w_offset(dims, l);
        double* Pl = P + w_offset(dims, l);
        for (int o = 0; o < dims[l + 1]; ++o)
          for (int i = 0; i < dims[l]; ++i) Pl[int64_t(o) * dims[l] + i] += d[o] * H[i];
        if (l == 0) break;
        for (int i = 0; i < dims[l]; ++i) {
          double s = 0.0;
          for (int o = 0; o < dims[l + 1]; ++o) s += Wl[int64_t(o) * dims[l] + i] * d[o];
          dn[i] = H[i] > 0.0 ? s : 0.0;
        }
        for (int i = 0; i < dims[l]; ++i) d[i] = dn[i];
      }
    }
  });
  for (int64_t p = 0; p < n_par; ++p) dW[p] = 0.0;
  for (int64_t c = 0; c < n_chunks; ++c)
    for (int64_t p = 0; p < n_par; ++p) dW[p] += part[c * n_par + p];
}

// ------------------------------------------------------ Sec. 5 "Optimizer" --
// Adam (Kingma & Ba 2015) step t >= 1 with bias correction.
void oracle_adam(double* W, double* m, double* v, const double* g, int64_t count, int64_t t, double lr, double b1,
                 double b2, double eps) {
  const double c1 = 1.0 - std::pow(b1, double(t));
  const double c2 = 1.0 - std::pow(b2, double(t));
  for (int64_t p = 0; p < count; ++p) {
    m[p] = b1 * m[p] + (1.0 - b1) * g[p];
    v[p] = b2 * v[p] + (1.0 - b2) * g[p] * g[p];
    const double mh = m[p] / c1;
    const double vh = v[p] / c2;
    W[p] -= lr * mh / (std::sqrt(vh) + eps);
  }
}

// ------------------------------------------- Sec. 3.3, Eq. 2 (as read) -----
// One update of the weight average after optimisation step t >= 1:
// EMA_t = ((1 - alpha) W_t + alpha eta_{t-1} EMA_{t-1}) / eta_t with
// eta_t = 1 - alpha^t (eta_0 = 0, so EMA_1 = W_1 whatever EMA_0 holds).
void oracle_ema(double* ema, const double* W, int64_t count, int64_t t, double alpha) {
  const double eta_t = 1.0 - std::pow(alpha, double(t));
  const double eta_prev = 1.0 - std::pow(alpha, double(t - 1));
  for (int64_t p = 0; p < count; ++p) ema[p] = ((1.0 - alpha) * W[p] + alpha * eta_prev * ema[p]) / eta_t;
}

// ------------------------------- Sec. 5 "Reflectance factorization" ---------
// Multiplies each row's 3 outputs by the record's diffuse + specular albedo
// (record floats 8..10 and 11..13), channel by channel.
void oracle_factor(const float* rec, int64_t n, double* y) {
  for (int64_t r = 0; r < n; ++r)
    for (int ch = 0; ch < 3; ++ch)
      y[r * 3 + ch] *= double(rec[r * kRecFloats + 8 + ch]) + double(rec[r * kRecFloats + 11 + ch]);
}

// ------------------------------------------------------------ composites ----
// Inference (Sec. 3.1: the cache is queried at terminal vertices): encode,
// then forward.
void oracle_infer(const double* W, const int* dims, int n_mats, const float* rec, int64_t n, int enc_mode,
                  double pad_value, int refl_factor, double* y) {
  std::vector<double> x(static_cast<size_t>(n) * kEncDims);
  oracle_encode(rec, n, enc_mode, pad_value, x.data());
  oracle_forward(W, dims, n_mats, x.data(), n, y, nullptr);
  if (refl_factor) oracle_factor(rec, n, y);
}

// One optimisation step (Sec. 3.3: several steps per frame, each on a disjoint
// slice of the shuffled records): gather, encode, forward, loss, backward,
// Adam.  W, m, v are updated in place; *t is incremented first (t counts
// steps from 1).  Returns the loss of the batch before the update; grad (if
// not null) receives dW.  With refl_factor the loss compares the factorised
// prediction y * f (f = diffuse + specular albedo) with the target, so the
// gradient reaching the network output is dL/d(y f) * f.
double oracle_train_step(double* W, double* m, double* v, int64_t* t, const int* dims, int n_mats, const float* pool,
                         const float* target, int64_t n_pool, int64_t batch, uint64_t frame_seed, int step,
                         int enc_mode, double pad_value, int loss_mode, double loss_eps, double lr, double b1,
                         double b2, double adam_eps, int refl_factor, double* grad) {
  std::vector<float> rec(static_cast<size_t>(batch) * kRecFloats);
  std::vector<float> tgt(static_cast<size_t>(batch) * 3);
  oracle_gather(pool, target, n_pool, batch, frame_seed, step, rec.data(), tgt.data(), nullptr);
  std::vector<double> x(static_cast<size_t>(batch) * kEncDims);
  oracle_encode(rec.data(), batch, enc_mode, pad_value, x.data());
  int64_t act_total = 0;
  for (int l = 0; l < n_mats; ++l) act_total += batch * dims[l];
  std::vector<double> acts(static_cast<size_t>(act_total));
  std::vector<double> y(static_cast<size_t>(batch) * dims[n_mats]);
  std::vector<double> g(static_cast<size_t>(batch) * dims[n_mats]);
  oracle_forward(W, dims, n_mats, x.data(), batch, y.data(), acts.data());
  if (refl_factor) oracle_factor(rec.data(), batch, y.data());
  const double loss = oracle_loss(y.data(), tgt.data(), batch, loss_mode, loss_eps, g.data());
  if (refl_factor) oracle_factor(rec.data(), batch, g.data());  // chain rule through y * f
  const int64_t n_par = w_offset(dims, n_mats);
  std::vector<double> dW(static_cast<size_t>(n_par));
  oracle_backward(W, dims, n_mats, acts.data(), g.data(), batch, dW.data());
  if (grad)
    for (int64_t p = 0; p < n_par; ++p) grad[p] = dW[p];
  *t += 1;
  oracle_adam(W, m, v, dW.data(), n_par, *t, lr, b1, b2, adam_eps);
  return loss;
}

}  // extern "C"

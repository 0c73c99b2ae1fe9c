// FP64 CPU oracle for shearlet-regularised convex multi-label segmentation
// (S. Haeuser, G. Steidl, "Convex Multiclass Segmentation with Shearlet
// Regularization", arXiv:1112.1805).
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
// includes this file; only the test suite, the smoke check and the CPU leg of
// the benchmark load it.  It shares no code with the CUDA path: it has its own
// FFT (recursive mixed-radix decimation in time, direct DFT for prime
// lengths), its own filter construction over the FULL frequency plane, its own
// transforms and its own ADMM that keeps v, b_v, w, b_w explicitly as the
// paper writes them.
//
// Conventions (readings of the paper, each one stated where it is used):
//   * images are row-major [H][W]; the first frequency coordinate omega_1
//     belongs to the row index (axis of length H), omega_2 to the column index;
//   * DFT index n in [0,N) stands for the frequency omega = n for n < ceil(N/2)
//     and omega = n - N otherwise (the set Omega of Sec. 2, "Finite Discrete
//     Shearlets");
//   * per axis the frequency is normalised as xi_a = omega_a * 4^J / N_a, so
//     that the J scales cover the band up to Nyquist for any (N, J);
//   * on the Nyquist lines of even-sized axes the DFT partner of a frequency is
//     not its continuous mirror; there each filter is replaced by the root mean
//     square of its values at the two partners, which keeps the partition of
//     unity and makes every coefficient of a real image real;
//   * filter order per label: low-pass; then for j = 0..J-1: horizontal-cone
//     shears k = -2^j+1..2^j-1, vertical-cone shears (same k), glued k = -2^j,
//     glued k = +2^j;  eta = 2^(J+2) - 3 filters in all;
//   * regularisation weights: Lambda[0] for the low-pass, Lambda[j+1] for
//     scale j.
//
// Parity status of each exported function is stated in its comment; the pins
// live in tests/test_oracle_*.py.

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <functional>
#include <thread>
#include <vector>

namespace {

using cd = std::complex<double>;
constexpr double kPi = 3.14159265358979323846264338327950288;

// ---------------------------------------------------------------------------
// 1-D windows, Sec. 2 "Continuous Shearlets" (Meyer construction).
// ---------------------------------------------------------------------------

// Auxiliary polynomial v: 0 below 0, 35x^4 - 84x^5 + 70x^6 - 20x^7 on [0,1],
// 1 above 1.
double meyer_v(double x) {
  if (x < 0.0) return 0.0;
  if (x > 1.0) return 1.0;
  const double x4 = x * x * x * x;
  return 35.0 * x4 - 84.0 * x4 * x + 70.0 * x4 * x * x - 20.0 * x4 * x * x * x;
}

// Radial Meyer window b: sin(pi/2 v(|x|-1)) on [1,2], cos(pi/2 v(|x|/2-1)) on
// (2,4], 0 elsewhere.
double meyer_b(double x) {
  const double a = std::fabs(x);
  if (a >= 1.0 && a <= 2.0) return std::sin(0.5 * kPi * meyer_v(a - 1.0));
  if (a > 2.0 && a <= 4.0) return std::cos(0.5 * kPi * meyer_v(0.5 * a - 1.0));
  return 0.0;
}

// psi1_hat(w) = sqrt(b(2w)^2 + b(w)^2)  (eq. psi1_psi2).
double psi1_hat(double w) {
  const double b2 = meyer_b(2.0 * w), b1 = meyer_b(w);
  return std::sqrt(b2 * b2 + b1 * b1);
}

// psi2_hat(w) = sqrt(v(1+w)) for w <= 0, sqrt(v(1-w)) for w > 0
// (eq. psi1_psi2).
double psi2_hat(double w) {
  return w <= 0.0 ? std::sqrt(meyer_v(1.0 + w)) : std::sqrt(meyer_v(1.0 - w));
}

// Low-pass profile varphi: 1 on |w| <= 1/2, cos(pi/2 v(2|w|-1)) on (1/2,1),
// 0 elsewhere (scaling function paragraph of Sec. 2).
double varphi(double w) {
  const double a = std::fabs(w);
  if (a <= 0.5) return 1.0;
  if (a < 1.0) return std::cos(0.5 * kPi * meyer_v(2.0 * a - 1.0));
  return 0.0;
}

int num_filters(int J) { return (1 << (J + 2)) - 3; }

// DFT index -> frequency in Omega = {-floor(N/2), ..., ceil(N/2)-1}.
long freq_of_index(long n, long N) { return n < (N + 1) / 2 ? n : n - N; }

// ---------------------------------------------------------------------------
// Filter bank, Sec. 2 "Finite Discrete Shearlets" and the glued seam
// shearlets; Theorem (Parseval frame).  Values before Nyquist symmetrisation.
// ---------------------------------------------------------------------------
struct FilterSpec {
  int kind;  // 0 low-pass, 1 horizontal cone, 2 vertical cone, 3 glued
  int j;     // scale
  int k;     // shear
};

std::vector<FilterSpec> filter_list(int J) {
  std::vector<FilterSpec> out;
  out.push_back({0, 0, 0});
  for (int j = 0; j < J; ++j) {
    const int p = 1 << j;
    for (int k = -p + 1; k <= p - 1; ++k) out.push_back({1, j, k});
    for (int k = -p + 1; k <= p - 1; ++k) out.push_back({2, j, k});
    out.push_back({3, j, -p});
    out.push_back({3, j, p});
  }
  return out;
}

// Shearlet value for the horizontal cone formula psi1(4^-j xi1) psi2(2^j xi2/xi1 + k)
// at integer frequency (w1, w2) of an H x W grid, xi_a = w_a 4^J / N_a.
double h_formula(long w1, long w2, long H, long W, int J, int j, int k) {
  const double x1 = static_cast<double>(w1) * std::ldexp(1.0, 2 * (J - j)) / static_cast<double>(H);
  const double ratio = static_cast<double>(w2 * H) / static_cast<double>(w1 * W);  // xi2 / xi1
  return psi1_hat(x1) * psi2_hat(std::ldexp(ratio, j) + static_cast<double>(k));
}

// Vertical cone formula: the roles of the two coordinates exchanged.
double v_formula(long w1, long w2, long H, long W, int J, int j, int k) {
  const double x2 = static_cast<double>(w2) * std::ldexp(1.0, 2 * (J - j)) / static_cast<double>(W);
  const double ratio = static_cast<double>(w1 * W) / static_cast<double>(w2 * H);  // xi1 / xi2
  return psi1_hat(x2) * psi2_hat(std::ldexp(ratio, j) + static_cast<double>(k));
}

double filter_value_raw(const FilterSpec& fs, long w1, long w2, long H, long W, int J) {
  // |xi1| versus |xi2| compared exactly in integers: |xi1| < |xi2| iff |w1| W < |w2| H.
  const long a1 = std::labs(w1) * W, a2 = std::labs(w2) * H;
  if (fs.kind == 0) {
    const double x1 = std::fabs(static_cast<double>(w1) * std::ldexp(1.0, 2 * J) / static_cast<double>(H));
    const double x2 = std::fabs(static_cast<double>(w2) * std::ldexp(1.0, 2 * J) / static_cast<double>(W));
    return varphi(std::max(x1, x2));
  }
  const bool in_h = a2 < a1;               // |xi2| < |xi1|   (cone C^h)
  const bool in_v = a1 < a2;               // |xi1| < |xi2|   (cone C^v)
  const bool on_seam = (a1 == a2) && a1 > 0;  // |xi1| = |xi2| (seam C^x)
  switch (fs.kind) {
    case 1: return in_h ? h_formula(w1, w2, H, W, J, fs.j, fs.k) : 0.0;
    case 2: return in_v ? v_formula(w1, w2, H, W, J, fs.j, fs.k) : 0.0;
    default:  // glued seam shearlet = h part + v part + seam part
      if (in_h) return h_formula(w1, w2, H, W, J, fs.j, fs.k);
      if (in_v) return v_formula(w1, w2, H, W, J, fs.j, fs.k);
      if (on_seam) return h_formula(w1, w2, H, W, J, fs.j, fs.k);
      return 0.0;
  }
}

// Full-plane filter bank [eta][H][W] in DFT index order, symmetrised on the
// Nyquist lines.
std::vector<double> build_filters(int H, int W, int J) {
  const auto specs = filter_list(J);
  const size_t P = static_cast<size_t>(H) * W;
  std::vector<double> out(specs.size() * P);
  for (size_t f = 0; f < specs.size(); ++f) {
    double* F = out.data() + f * P;
    for (long n1 = 0; n1 < H; ++n1)
      for (long n2 = 0; n2 < W; ++n2)
        F[n1 * W + n2] = filter_value_raw(specs[f], freq_of_index(n1, H), freq_of_index(n2, W), H, W, J);
    // Nyquist symmetrisation: the DFT partner of (n1, n2) is (-n1 mod H, -n2 mod W).
    std::vector<double> G(F, F + P);
    for (long n1 = 0; n1 < H; ++n1)
      for (long n2 = 0; n2 < W; ++n2) {
        const bool nyq = (H % 2 == 0 && n1 == H / 2) || (W % 2 == 0 && n2 == W / 2);
        if (!nyq) continue;
        const long m1 = (H - n1) % H, m2 = (W - n2) % W;
        const double a = G[n1 * W + n2], b = G[m1 * W + m2];
        F[n1 * W + n2] = std::sqrt(0.5 * (a * a + b * b));
      }
  }
  return out;
}

// ---------------------------------------------------------------------------
// FFT (Sec. 2: fft2 without normalisation, ifft2 with 1/(H W)).
// Recursive mixed-radix decimation in time: x[p t + r] is split into p
// sub-sequences of length n/p, transformed, and combined with the twiddles
// exp(sign 2 pi i r q / n).  Prime lengths use the direct DFT.
// ---------------------------------------------------------------------------
int smallest_prime_factor(int n) {
  for (int p = 2; p * p <= n; ++p)
    if (n % p == 0) return p;
  return n;
}

// out[q] = sum_t in[t*stride] exp(sign 2 pi i t q / n), q < n.  roots[m] =
// exp(sign 2 pi i m / N) for the top-level length N (n divides N); scratch has
// room for n values.
void fft_rec(const cd* in, size_t stride, cd* out, int n, const cd* roots, int N, cd* scratch) {
  if (n == 1) {
    out[0] = in[0];
    return;
  }
  const int p = smallest_prime_factor(n);
  const int step = N / n;
  if (p == n) {
    for (int q = 0; q < n; ++q) {
      cd acc = 0.0;
      for (int t = 0; t < n; ++t) acc += in[t * stride] * roots[(static_cast<long>(t) * q % n) * step];
      scratch[q] = acc;
    }
    std::copy(scratch, scratch + n, out);
    return;
  }
  const int m = n / p;
  for (int r = 0; r < p; ++r) fft_rec(in + r * stride, stride * p, out + r * m, m, roots, N, scratch);
  for (int q = 0; q < n; ++q) {
    cd acc = 0.0;
    for (int r = 0; r < p; ++r) acc += roots[(static_cast<long>(r) * q % n) * step] * out[r * m + q % m];
    scratch[q] = acc;
  }
  std::copy(scratch, scratch + n, out);
}

std::vector<cd> roots_of_unity(int N, int sign) {
  std::vector<cd> r(N);
  for (int m = 0; m < N; ++m) {
    const double ang = sign * 2.0 * kPi * static_cast<double>(m) / static_cast<double>(N);
    r[m] = cd(std::cos(ang), std::sin(ang));
  }
  return r;
}

// In-place 2-D DFT of an H x W complex array.  inverse=false: exponent -1, no
// scaling (fft2); inverse=true: exponent +1 and factor 1/(H W) (ifft2).
void fft2(cd* a, int H, int W, bool inverse) {
  const int sign = inverse ? +1 : -1;
  const auto rW = roots_of_unity(W, sign), rH = roots_of_unity(H, sign);
  std::vector<cd> tmp(std::max(H, W)), out(std::max(H, W)), scratch(std::max(H, W));
  for (int r = 0; r < H; ++r) {
    fft_rec(a + static_cast<size_t>(r) * W, 1, out.data(), W, rW.data(), W, scratch.data());
    std::copy(out.begin(), out.begin() + W, a + static_cast<size_t>(r) * W);
  }
  for (int c = 0; c < W; ++c) {
    for (int r = 0; r < H; ++r) tmp[r] = a[static_cast<size_t>(r) * W + c];
    fft_rec(tmp.data(), 1, out.data(), H, rH.data(), H, scratch.data());
    for (int r = 0; r < H; ++r) a[static_cast<size_t>(r) * W + c] = out[r];
  }
  if (inverse) {
    const double s = 1.0 / (static_cast<double>(H) * W);
    for (size_t i = 0; i < static_cast<size_t>(H) * W; ++i) a[i] *= s;
  }
}

// ---------------------------------------------------------------------------
// Threads: a plain parallel-for over independent work items.
// ---------------------------------------------------------------------------
int g_threads = 0;

int thread_count() {
  if (g_threads > 0) return g_threads;
  const unsigned hc = std::thread::hardware_concurrency();
  return hc ? static_cast<int>(hc) : 1;
}

void parallel_for(int n, const std::function<void(int)>& body) {
  const int nt = std::min(thread_count(), n);
  if (nt <= 1) {
    for (int i = 0; i < n; ++i) body(i);
    return;
  }
  std::vector<std::thread> pool;
  for (int t = 0; t < nt; ++t)
    pool.emplace_back([&, t] {
      for (int i = t; i < n; i += nt) body(i);
    });
  for (auto& th : pool) th.join();
}

// ---------------------------------------------------------------------------
// Shearlet transform S and its adjoint S^T (eq. wichtig; synthesis paragraph
// after the Theorem).  Filters F are the full-plane bank.
// ---------------------------------------------------------------------------
struct Transform {
  int H, W, J, eta;
  std::vector<double> F;  // [eta][H][W]
  Transform(int H_, int W_, int J_) : H(H_), W(W_), J(J_), eta(num_filters(J_)), F(build_filters(H_, W_, J_)) {}
  size_t P() const { return static_cast<size_t>(H) * W; }
};

// coef[f][H][W] = ifft2(F_f . fft2(u)) for one channel; returns the largest
// |imaginary part| met (the real part is kept).
double analyze_one(const Transform& T, const double* u, double* coef) {
  const size_t P = T.P();
  std::vector<cd> U(P), G(P);
  for (size_t i = 0; i < P; ++i) U[i] = u[i];
  fft2(U.data(), T.H, T.W, false);
  double max_im = 0.0;
  for (int f = 0; f < T.eta; ++f) {
    const double* F = T.F.data() + static_cast<size_t>(f) * P;
    for (size_t i = 0; i < P; ++i) G[i] = F[i] * U[i];
    fft2(G.data(), T.H, T.W, true);
    for (size_t i = 0; i < P; ++i) {
      coef[static_cast<size_t>(f) * P + i] = G[i].real();
      max_im = std::max(max_im, std::fabs(G[i].imag()));
    }
  }
  return max_im;
}

// u = ifft2( sum_f F_f . fft2(coef_f) ) for one channel.
double synthesize_one(const Transform& T, const double* coef, double* u) {
  const size_t P = T.P();
  std::vector<cd> acc(P, 0.0), G(P);
  for (int f = 0; f < T.eta; ++f) {
    const double* F = T.F.data() + static_cast<size_t>(f) * P;
    for (size_t i = 0; i < P; ++i) G[i] = coef[static_cast<size_t>(f) * P + i];
    fft2(G.data(), T.H, T.W, false);
    for (size_t i = 0; i < P; ++i) acc[i] += F[i] * G[i];
  }
  fft2(acc.data(), T.H, T.W, true);
  double max_im = 0.0;
  for (size_t i = 0; i < P; ++i) {
    u[i] = acc[i].real();
    max_im = std::max(max_im, std::fabs(acc[i].imag()));
  }
  return max_im;
}

// Per-(channel, filter) parallel analysis: one forward FFT per channel, then
// the eta filtered inverse FFTs spread over threads.
double analyze_many(const Transform& T, const double* u, int nch, double* coef) {
  const size_t P = T.P();
  std::vector<std::vector<cd>> U(nch, std::vector<cd>(P));
  parallel_for(nch, [&](int c) {
    for (size_t i = 0; i < P; ++i) U[c][i] = u[static_cast<size_t>(c) * P + i];
    fft2(U[c].data(), T.H, T.W, false);
  });
  std::vector<double> max_im(static_cast<size_t>(nch) * T.eta, 0.0);
  parallel_for(nch * T.eta, [&](int item) {
    const int c = item / T.eta, f = item % T.eta;
    const double* F = T.F.data() + static_cast<size_t>(f) * P;
    std::vector<cd> G(P);
    for (size_t i = 0; i < P; ++i) G[i] = F[i] * U[c][i];
    fft2(G.data(), T.H, T.W, true);
    double* out = coef + (static_cast<size_t>(c) * T.eta + f) * P;
    double m = 0.0;
    for (size_t i = 0; i < P; ++i) {
      out[i] = G[i].real();
      m = std::max(m, std::fabs(G[i].imag()));
    }
    max_im[item] = m;
  });
  return *std::max_element(max_im.begin(), max_im.end());
}

// Parallel synthesis: the forward FFT of every coefficient image in parallel,
// then the filter-weighted sum per channel in filter order, one inverse FFT.
double synthesize_many(const Transform& T, const double* coef, int nch, double* u) {
  const size_t P = T.P();
  std::vector<std::vector<cd>> G(static_cast<size_t>(nch) * T.eta);
  parallel_for(nch * T.eta, [&](int item) {
    auto& g = G[item];
    g.resize(P);
    const double* in = coef + static_cast<size_t>(item) * P;
    for (size_t i = 0; i < P; ++i) g[i] = in[i];
    fft2(g.data(), T.H, T.W, false);
  });
  std::vector<double> max_im(nch, 0.0);
  parallel_for(nch, [&](int c) {
    std::vector<cd> acc(P, 0.0);
    for (int f = 0; f < T.eta; ++f) {
      const double* F = T.F.data() + static_cast<size_t>(f) * P;
      const auto& g = G[static_cast<size_t>(c) * T.eta + f];
      for (size_t i = 0; i < P; ++i) acc[i] += F[i] * g[i];
    }
    fft2(acc.data(), T.H, T.W, true);
    double m = 0.0;
    for (size_t i = 0; i < P; ++i) {
      u[static_cast<size_t>(c) * P + i] = acc[i].real();
      m = std::max(m, std::fabs(acc[i].imag()));
    }
    max_im[c] = m;
  });
  return *std::max_element(max_im.begin(), max_im.end());
}

// ---------------------------------------------------------------------------
// Proximal maps of Sec. 3 (ADMM paragraph).
// ---------------------------------------------------------------------------

// Soft shrinkage S_t(x): x - t for x > t, 0 on [-t, t], x + t for x < -t.
double soft_shrink(double x, double t) {
  if (x > t) return x - t;
  if (x < -t) return x + t;
  return 0.0;
}

// Euclidean projection onto the unit simplex {x >= 0, sum x = 1} by sorting:
// with y sorted descending, rho = max{r : y_r - (sum_{i<=r} y_i - 1)/r > 0},
// tau = (sum_{i<=rho} y_i - 1)/rho, x = max(g - tau, 0).
void project_simplex_sort(const double* g, int K, double* x) {
  std::vector<double> y(g, g + K);
  std::sort(y.begin(), y.end(), std::greater<double>());
  double cum = 0.0, tau = 0.0;
  for (int r = 0; r < K; ++r) {
    cum += y[r];
    const double t = (cum - 1.0) / (r + 1);
    if (y[r] - t > 0.0) tau = t;
  }
  for (int k = 0; k < K; ++k) x[k] = std::max(g[k] - tau, 0.0);
}

// The paper's own description: project onto the hyperplane sum x = 1 by
// g~ = g + (1 - sum g)/q * 1, set the negative components to zero, project the
// remaining ones again onto the hyperplane of the lower-dimensional space, and
// repeat until no component is negative.
void project_simplex_repeated(const double* g, int K, double* x) {
  std::vector<bool> active(K, true);
  std::vector<double> y(g, g + K);
  for (int pass = 0; pass <= K; ++pass) {
    int q = 0;
    double sum = 0.0;
    for (int k = 0; k < K; ++k)
      if (active[k]) {
        ++q;
        sum += g[k];
      }
    const double shift = (1.0 - sum) / q;
    bool changed = false;
    for (int k = 0; k < K; ++k) {
      if (!active[k]) {
        y[k] = 0.0;
        continue;
      }
      y[k] = g[k] + shift;
      if (y[k] < 0.0) {
        active[k] = false;
        changed = true;
      }
    }
    if (!changed) break;
  }
  for (int k = 0; k < K; ++k) x[k] = active[k] ? y[k] : 0.0;
}

}  // namespace

// ===========================================================================
// Exported C interface (ctypes).  All arrays are host FP64, row-major.
// Return 0 on success, -1 on an argument error.
// ===========================================================================
extern "C" {

// Threads used by the parallel loops (0 = all hardware threads).
void oracle_set_threads(int n) { g_threads = n; }
int oracle_get_threads(void) { return thread_count(); }

// eta = 2^(J+2) - 3 (Remark 1: 61 images for 4 scales).
int oracle_num_filters(int J) { return J >= 1 ? num_filters(J) : -1; }

// Vectorised 1-D windows for the pins of Sec. 2 (which: 0 v, 1 b, 2 psi1_hat,
// 3 psi2_hat, 4 varphi).
int oracle_window(int which, const double* x, long n, double* y) {
  for (long i = 0; i < n; ++i) {
    switch (which) {
      case 0: y[i] = meyer_v(x[i]); break;
      case 1: y[i] = meyer_b(x[i]); break;
      case 2: y[i] = psi1_hat(x[i]); break;
      case 3: y[i] = psi2_hat(x[i]); break;
      case 4: y[i] = varphi(x[i]); break;
      default: return -1;
    }
  }
  return 0;
}

// Filter descriptors (kind, j, k) in bank order, 3 ints per filter.
int oracle_filter_specs(int J, int* out) {
  if (J < 1) return -1;
  const auto s = filter_list(J);
  for (size_t f = 0; f < s.size(); ++f) {
    out[3 * f] = s[f].kind;
    out[3 * f + 1] = s[f].j;
    out[3 * f + 2] = s[f].k;
  }
  return 0;
}

// Full-plane filter bank out[eta][H][W] (Sec. 2 finite discrete shearlets).
int oracle_filters(int H, int W, int J, double* out) {
  if (H < 2 || W < 2 || J < 1) return -1;
  const auto F = build_filters(H, W, J);
  std::memcpy(out, F.data(), F.size() * sizeof(double));
  return 0;
}

// Filter bank without the Nyquist symmetrisation (for the pin that shows why
// the symmetrisation is needed).
int oracle_filters_unsymmetrised(int H, int W, int J, double* out) {
  if (H < 2 || W < 2 || J < 1) return -1;
  const auto specs = filter_list(J);
  const size_t P = static_cast<size_t>(H) * W;
  for (size_t f = 0; f < specs.size(); ++f)
    for (long n1 = 0; n1 < H; ++n1)
      for (long n2 = 0; n2 < W; ++n2)
        out[f * P + n1 * W + n2] =
            filter_value_raw(specs[f], freq_of_index(n1, H), freq_of_index(n2, W), H, W, J);
  return 0;
}

// 2-D DFT of interleaved complex data (re, im) [H][W][2] with the oracle's own
// FFT; inverse != 0 gives ifft2 (with 1/(HW)).
int oracle_fft2(int H, int W, const double* in, double* out, int inverse) {
  if (H < 1 || W < 1) return -1;
  std::vector<cd> a(static_cast<size_t>(H) * W);
  for (size_t i = 0; i < a.size(); ++i) a[i] = cd(in[2 * i], in[2 * i + 1]);
  fft2(a.data(), H, W, inverse != 0);
  for (size_t i = 0; i < a.size(); ++i) {
    out[2 * i] = a[i].real();
    out[2 * i + 1] = a[i].imag();
  }
  return 0;
}

// Brute-force 2-D DFT by the defining double sum (the pin for oracle_fft2).
int oracle_dft2_brute(int H, int W, const double* in, double* out, int inverse) {
  if (H < 1 || W < 1) return -1;
  const double sign = inverse ? +1.0 : -1.0;
  for (int a = 0; a < H; ++a)
    for (int b = 0; b < W; ++b) {
      cd acc = 0.0;
      for (int m1 = 0; m1 < H; ++m1)
        for (int m2 = 0; m2 < W; ++m2) {
          const double ang = sign * 2.0 * kPi *
                             (static_cast<double>((static_cast<long>(a) * m1) % H) / H +
                              static_cast<double>((static_cast<long>(b) * m2) % W) / W);
          acc += cd(in[2 * (m1 * W + m2)], in[2 * (m1 * W + m2) + 1]) * cd(std::cos(ang), std::sin(ang));
        }
      if (inverse) acc /= static_cast<double>(H) * W;
      out[2 * (a * W + b)] = acc.real();
      out[2 * (a * W + b) + 1] = acc.imag();
    }
  return 0;
}

// Analysis S (eq. wichtig): coef[c][f][H][W] from u[c][H][W].  *max_imag gets
// the largest imaginary part discarded.
int oracle_analyze(int H, int W, int J, const double* u, int nch, double* coef, double* max_imag) {
  if (H < 2 || W < 2 || J < 1 || nch < 1) return -1;
  Transform T(H, W, J);
  const double m = analyze_many(T, u, nch, coef);
  if (max_imag) *max_imag = m;
  return 0;
}

// Synthesis S^T (inverse shearlet transform, Fourier-domain form after the
// Theorem): u[c][H][W] from coef[c][f][H][W].
int oracle_synthesize(int H, int W, int J, const double* coef, int nch, double* u, double* max_imag) {
  if (H < 2 || W < 2 || J < 1 || nch < 1) return -1;
  Transform T(H, W, J);
  const double m = synthesize_many(T, coef, nch, u);
  if (max_imag) *max_imag = m;
  return 0;
}

// Data term, eq. computationOfs with p = 2 and its RGB form:
// s[k][r] = sum_ch (f[ch][r] - c[k][ch])^2.
int oracle_data_term(int H, int W, int C, const double* f, int K, const double* codebook, double* s) {
  if (H < 1 || W < 1 || C < 1 || K < 1) return -1;
  const size_t P = static_cast<size_t>(H) * W;
  for (int k = 0; k < K; ++k)
    for (size_t r = 0; r < P; ++r) {
      double acc = 0.0;
      for (int ch = 0; ch < C; ++ch) {
        const double d = f[ch * P + r] - codebook[k * C + ch];
        acc += d * d;
      }
      s[k * P + r] = acc;
    }
  return 0;
}

// Soft shrinkage, elementwise.
int oracle_soft_shrink(const double* x, long n, double t, double* y) {
  for (long i = 0; i < n; ++i) y[i] = soft_shrink(x[i], t);
  return 0;
}

// Simplex projection of `count` vectors of length K (method 0: sorting,
// method 1: the paper's repeated hyperplane projection).
int oracle_project_simplex(const double* g, long count, int K, double* x, int method) {
  if (K < 1) return -1;
  for (long i = 0; i < count; ++i) {
    if (method == 0)
      project_simplex_sort(g + i * K, K, x + i * K);
    else
      project_simplex_repeated(g + i * K, K, x + i * K);
  }
  return 0;
}

// T iterations of the ADMM of Sec. 3 for problem (eq. problemSegmentationADMM),
// in place on the state (v, bv: [K][eta][H][W]; w, bw, u: [K][H][W]).  One
// iteration, with gamma > 0 and thresholds gamma*Lambda per scale:
//   u   = 1/2 [ S^T (v - b_v) + (w - b_w) - gamma s ]      (u-step, A^T A = 2I)
//   g_v = b_v + S u ;  v = S_{gamma Lambda}(g_v)           (v-step)
//   g_w = b_w + u   ;  w = P_C(g_w) pixelwise              (w-step)
//   b_v = g_v - v   ;  b_w = g_w - w                       (b-update)
// fp_res (nullable, length T) receives, per iteration, the fixed-point residual
// ||v+ - v||^2 + ||w+ - w||^2 + ||b_v+ - b_v||^2 + ||b_w+ - b_w||^2.
// proj_method: 0 sorting, 1 repeated hyperplane projection.
int oracle_admm_iterate(int H, int W, int J, int K, const double* s, const double* Lambda, double gamma, int T,
                        double* v, double* bv, double* w, double* bw, double* u, double* fp_res,
                        int proj_method) {
  if (H < 2 || W < 2 || J < 1 || K < 1 || T < 0 || !(gamma > 0.0)) return -1;
  Transform Tr(H, W, J);
  const int eta = Tr.eta;
  const size_t P = Tr.P();
  const size_t NC = static_cast<size_t>(K) * eta * P;
  const auto specs = filter_list(J);
  std::vector<double> thr(eta);
  for (int f = 0; f < eta; ++f) thr[f] = gamma * (specs[f].kind == 0 ? Lambda[0] : Lambda[specs[f].j + 1]);

  std::vector<double> diff(NC), st(static_cast<size_t>(K) * P), su(NC);
  for (int it = 0; it < T; ++it) {
    // u-step
    for (size_t i = 0; i < NC; ++i) diff[i] = v[i] - bv[i];
    synthesize_many(Tr, diff.data(), K, st.data());
    for (size_t i = 0; i < static_cast<size_t>(K) * P; ++i) u[i] = 0.5 * (st[i] + (w[i] - bw[i]) - gamma * s[i]);
    // v-step and b_v
    analyze_many(Tr, u, K, su.data());
    double res = 0.0;
    for (int k = 0; k < K; ++k)
      for (int f = 0; f < eta; ++f) {
        const size_t base = (static_cast<size_t>(k) * eta + f) * P;
        for (size_t r = 0; r < P; ++r) {
          const double gv = bv[base + r] + su[base + r];
          const double vn = soft_shrink(gv, thr[f]);
          const double bn = gv - vn;
          res += (vn - v[base + r]) * (vn - v[base + r]) + (bn - bv[base + r]) * (bn - bv[base + r]);
          v[base + r] = vn;
          bv[base + r] = bn;
        }
      }
    // w-step and b_w, pixelwise over the K labels
    std::vector<double> g(K), x(K);
    for (size_t r = 0; r < P; ++r) {
      for (int k = 0; k < K; ++k) g[k] = bw[k * P + r] + u[k * P + r];
      if (proj_method == 0)
        project_simplex_sort(g.data(), K, x.data());
      else
        project_simplex_repeated(g.data(), K, x.data());
      for (int k = 0; k < K; ++k) {
        const double bn = g[k] - x[k];
        res += (x[k] - w[k * P + r]) * (x[k] - w[k * P + r]) + (bn - bw[k * P + r]) * (bn - bw[k * P + r]);
        w[k * P + r] = x[k];
        bw[k * P + r] = bn;
      }
    }
    if (fp_res) fp_res[it] = res;
  }
  return 0;
}

// Reverse mode of T iterations of oracle_admm_iterate from the zero state
// (the unrolled solve), for a given adjoint wbar_T of the final w.  Each
// iteration maps (b_v, Q = S^T(v - b_v), w, b_w) to its successor:
//   u = (Q + w - b_w - gamma s)/2,  g = b_v + S u,  b_v' = clip(g, t_f),
//   Q' = S^T (g - 2 clip(g, t_f)),  g_w = b_w + u,  w' = P_C(g_w),  b_w' = g_w - w',
// with t_f = gamma Lambda_{j(f)}.  Going backwards through one iteration:
//   gbar_w = bwbar' + J_P (wbar' - bwbar')   (J_P: projection onto the active
//            face, x_A - mean_A(x) on the support A of w', 0 elsewhere)
//   dbar = S Qbar'
//   gbar = dbar (1 - 2 m) + bvbar' m          (m = [|g| < t_f])
//   tbar_f += sum sign(g) (1 - m) (bvbar' - 2 dbar)
//   ubar = gbar_w + S^T gbar
//   Qbar = ubar/2, wbar = ubar/2, bwbar = gbar_w - ubar/2, bvbar = gbar,
//   sbar += -gamma ubar / 2.
// Outputs: sbar [K][H][W] (adjoint of the data term) and Lambar [J+1]
// (Lambar_j = gamma * sum of tbar_f over the filters of weight j).  The
// forward states are kept for all T iterations (test sizes only).
int oracle_unrolled_vjp(int H, int W, int J, int K, const double* s, const double* Lambda, double gamma, int T,
                        const double* wbar_T, double* sbar, double* Lambar, double* wT_out) {
  if (H < 2 || W < 2 || J < 1 || K < 1 || T < 1 || !(gamma > 0.0)) return -1;
  Transform Tr(H, W, J);
  const int eta = Tr.eta;
  const size_t P = Tr.P(), KP = static_cast<size_t>(K) * P, NC = static_cast<size_t>(K) * eta * P;
  const auto specs = filter_list(J);
  std::vector<double> thr(eta);
  for (int f = 0; f < eta; ++f) thr[f] = gamma * (specs[f].kind == 0 ? Lambda[0] : Lambda[specs[f].j + 1]);
  // forward, recording g (per coefficient) and w' (per pixel) of every iteration
  std::vector<double> bv(NC, 0.0), Q(KP, 0.0), w(KP, 0.0), bw(KP, 0.0), u(KP), c(NC), d(NC);
  std::vector<std::vector<double>> G(T), Wn(T);
  for (int it = 0; it < T; ++it) {
    for (size_t i = 0; i < KP; ++i) u[i] = 0.5 * (Q[i] + w[i] - bw[i] - gamma * s[i]);
    analyze_many(Tr, u.data(), K, c.data());
    G[it].resize(NC);
    for (int k = 0; k < K; ++k)
      for (int f = 0; f < eta; ++f) {
        const size_t base = (static_cast<size_t>(k) * eta + f) * P;
        for (size_t r = 0; r < P; ++r) {
          const double g = bv[base + r] + c[base + r];
          const double cl = std::min(std::max(g, -thr[f]), thr[f]);
          G[it][base + r] = g;
          bv[base + r] = cl;
          d[base + r] = g - 2.0 * cl;
        }
      }
    synthesize_many(Tr, d.data(), K, Q.data());
    std::vector<double> gw(K), x(K);
    for (size_t r = 0; r < P; ++r) {
      for (int k = 0; k < K; ++k) gw[k] = bw[k * P + r] + u[k * P + r];
      project_simplex_sort(gw.data(), K, x.data());
      for (int k = 0; k < K; ++k) {
        w[k * P + r] = x[k];
        bw[k * P + r] = gw[k] - x[k];
      }
    }
    Wn[it] = w;
  }
  if (wT_out) std::copy(w.begin(), w.end(), wT_out);
  // reverse
  std::vector<double> bvb(NC, 0.0), Qb(KP, 0.0), wb(wbar_T, wbar_T + KP), bwb(KP, 0.0), gwb(KP), ub(KP), db(NC),
      st(KP), tb(eta, 0.0);
  std::fill(sbar, sbar + KP, 0.0);
  for (int it = T - 1; it >= 0; --it) {
    const std::vector<double>& wn = Wn[it];
    for (size_t r = 0; r < P; ++r) {
      int q = 0;
      double mean = 0.0;
      for (int k = 0; k < K; ++k)
        if (wn[k * P + r] > 0.0) {
          ++q;
          mean += wb[k * P + r] - bwb[k * P + r];
        }
      mean /= q;
      for (int k = 0; k < K; ++k) {
        const double a = wb[k * P + r] - bwb[k * P + r];
        gwb[k * P + r] = bwb[k * P + r] + (wn[k * P + r] > 0.0 ? a - mean : 0.0);
      }
    }
    analyze_many(Tr, Qb.data(), K, db.data());
    for (int k = 0; k < K; ++k)
      for (int f = 0; f < eta; ++f) {
        const size_t base = (static_cast<size_t>(k) * eta + f) * P;
        double acc = 0.0;
        for (size_t r = 0; r < P; ++r) {
          const double g = G[it][base + r];
          const bool inside = std::fabs(g) < thr[f];
          const double gb = inside ? bvb[base + r] - db[base + r] : db[base + r];
          if (!inside) acc += (g > 0 ? 1.0 : -1.0) * (bvb[base + r] - 2.0 * db[base + r]);
          bvb[base + r] = gb;
        }
        tb[f] += acc;
      }
    synthesize_many(Tr, bvb.data(), K, st.data());
    for (size_t i = 0; i < KP; ++i) {
      ub[i] = gwb[i] + st[i];
      Qb[i] = 0.5 * ub[i];
      wb[i] = 0.5 * ub[i];
      bwb[i] = gwb[i] - 0.5 * ub[i];
      sbar[i] += -0.5 * gamma * ub[i];
    }
  }
  for (int j = 0; j <= J; ++j) Lambar[j] = 0.0;
  for (int f = 0; f < eta; ++f) Lambar[specs[f].kind == 0 ? 0 : specs[f].j + 1] += gamma * tb[f];
  return 0;
}

// Energy of eq. problemSegmentation at x: <x, s> + sum_f Lambda_{j(f)} ||(S x)_f||_1.
int oracle_energy(int H, int W, int J, int K, const double* x, const double* s, const double* Lambda, double* energy) {
  if (H < 2 || W < 2 || J < 1 || K < 1) return -1;
  Transform Tr(H, W, J);
  const size_t P = Tr.P();
  const auto specs = filter_list(J);
  std::vector<double> coef(static_cast<size_t>(K) * Tr.eta * P);
  analyze_many(Tr, x, K, coef.data());
  double data = 0.0, reg = 0.0;
  for (size_t i = 0; i < static_cast<size_t>(K) * P; ++i) data += x[i] * s[i];
  for (int k = 0; k < K; ++k)
    for (int f = 0; f < Tr.eta; ++f) {
      const double lam = specs[f].kind == 0 ? Lambda[0] : Lambda[specs[f].j + 1];
      double l1 = 0.0;
      const double* c = coef.data() + (static_cast<size_t>(k) * Tr.eta + f) * P;
      for (size_t r = 0; r < P; ++r) l1 += std::fabs(c[r]);
      reg += lam * l1;
    }
  *energy = data + reg;
  return 0;
}

// Label map: the index of the largest entry per pixel (ties: lowest index),
// and the gap between the largest and second largest entries.
int oracle_labels(int H, int W, int K, const double* x, int* labels, double* gap) {
  if (H < 1 || W < 1 || K < 1) return -1;
  const size_t P = static_cast<size_t>(H) * W;
  for (size_t r = 0; r < P; ++r) {
    int best = 0;
    double b1 = x[r], b2 = -INFINITY;
    for (int k = 1; k < K; ++k) {
      const double val = x[k * P + r];
      if (val > b1) {
        b2 = b1;
        b1 = val;
        best = k;
      } else if (val > b2) {
        b2 = val;
      }
    }
    labels[r] = best;
    if (gap) gap[r] = K > 1 ? b1 - b2 : INFINITY;
  }
  return 0;
}

}  // extern "C"

// ===========================================================================
// TV-regularised segmentation, the comparison model of Sec. 4 (eq. TVreg):
//   min_u <u, s> + lambda || |(I_q (x) grad) u| ||_1 + iota_C(u),
// with |(I_q (x) grad) u|(x) = (|grad u_1(x)|^2 + ... + |grad u_q(x)|^2)^(1/2)
// (the labels coupled per pixel), or, in the alternative the paper mentions,
// sum_k |grad u_k(x)|.  Readings (the paper states neither): grad is the
// forward difference with periodic boundary, the same periodic setting as the
// FFT-based shearlets, so that I + grad^T grad is diagonalised by the DFT; the
// ADMM is the one of Sec. 3 with S replaced by grad (same splitting v =
// (I_q (x) grad) u, w = u, same scaling by gamma), so that the u-step solves
// (I + grad^T grad) u = grad^T (v - b_v) + (w - b_w) - gamma s.
// Layout: gradients and their duals are [K][2][H][W], component 0 along the
// row axis (index r, omega_1), component 1 along the column axis.
// ===========================================================================
namespace {

// (grad u)(r, c) = (u(r+1, c) - u(r, c), u(r, c+1) - u(r, c)), periodic.
void tv_grad(int H, int W, const double* u, double* g) {
  const size_t P = static_cast<size_t>(H) * W;
  for (int r = 0; r < H; ++r)
    for (int c = 0; c < W; ++c) {
      const double x = u[r * W + c];
      g[r * W + c] = u[((r + 1) % H) * W + c] - x;
      g[P + r * W + c] = u[r * W + (c + 1) % W] - x;
    }
}

// Adjoint of tv_grad: (grad^T p)(r, c) = p0(r-1, c) - p0(r, c) + p1(r, c-1) - p1(r, c).
void tv_grad_adj(int H, int W, const double* p, double* out) {
  const size_t P = static_cast<size_t>(H) * W;
  for (int r = 0; r < H; ++r)
    for (int c = 0; c < W; ++c)
      out[r * W + c] = p[((r + H - 1) % H) * W + c] - p[r * W + c] + p[P + r * W + (c + W - 1) % W] - p[P + r * W + c];
}

// u = (I + grad^T grad)^(-1) rhs for one plane: grad^T grad is the periodic
// 5-point negative Laplacian, whose DFT symbol at index (n1, n2) is
// 4 sin^2(pi n1 / H) + 4 sin^2(pi n2 / W).
void tv_solve_one(int H, int W, const double* rhs, double* u) {
  const size_t P = static_cast<size_t>(H) * W;
  std::vector<cd> a(P);
  for (size_t i = 0; i < P; ++i) a[i] = rhs[i];
  fft2(a.data(), H, W, false);
  for (int n1 = 0; n1 < H; ++n1) {
    const double s1 = std::sin(kPi * n1 / H);
    for (int n2 = 0; n2 < W; ++n2) {
      const double s2 = std::sin(kPi * n2 / W);
      a[static_cast<size_t>(n1) * W + n2] /= 1.0 + 4.0 * s1 * s1 + 4.0 * s2 * s2;
    }
  }
  fft2(a.data(), H, W, true);
  for (size_t i = 0; i < P; ++i) u[i] = a[i].real();
}

// Proximal map of t |.|_2 on a group of n values: x (1 - t/|x|)_+.
void shrink_group(const double* x, int n, size_t stride, double t, double* out) {
  double nrm2 = 0.0;
  for (int i = 0; i < n; ++i) nrm2 += x[i * stride] * x[i * stride];
  const double nrm = std::sqrt(nrm2);
  const double f = nrm > t ? 1.0 - t / nrm : 0.0;
  for (int i = 0; i < n; ++i) out[i * stride] = f * x[i * stride];
}

// Vector shrinkage of g [K][2][H][W] with threshold t per pixel: the group is
// all 2K values of a pixel (per_label = 0, the coupled TV of eq. TVreg) or the
// two values of each label (per_label = 1).
void tv_shrink(int H, int W, int K, const double* g, double t, int per_label, double* v) {
  const size_t P = static_cast<size_t>(H) * W;
  for (size_t x = 0; x < P; ++x) {
    if (per_label) {
      for (int k = 0; k < K; ++k) shrink_group(g + 2 * k * P + x, 2, P, t, v + 2 * k * P + x);
    } else {
      shrink_group(g + x, 2 * K, P, t, v + x);
    }
  }
}

}  // namespace

extern "C" {

// grad u for K planes: u [K][H][W] -> g [K][2][H][W].
int oracle_tv_grad(int H, int W, int K, const double* u, double* g) {
  if (H < 2 || W < 2 || K < 1) return -1;
  const size_t P = static_cast<size_t>(H) * W;
  for (int k = 0; k < K; ++k) tv_grad(H, W, u + k * P, g + 2 * k * P);
  return 0;
}

// grad^T p for K planes: p [K][2][H][W] -> out [K][H][W].
int oracle_tv_grad_adj(int H, int W, int K, const double* p, double* out) {
  if (H < 2 || W < 2 || K < 1) return -1;
  const size_t P = static_cast<size_t>(H) * W;
  for (int k = 0; k < K; ++k) tv_grad_adj(H, W, p + 2 * k * P, out + k * P);
  return 0;
}

// (I + grad^T grad)^(-1) rhs for K planes.
int oracle_tv_solve(int H, int W, int K, const double* rhs, double* u) {
  if (H < 2 || W < 2 || K < 1) return -1;
  const size_t P = static_cast<size_t>(H) * W;
  parallel_for(K, [&](int k) { tv_solve_one(H, W, rhs + k * P, u + k * P); });
  return 0;
}

// Vector shrinkage (see tv_shrink), g and v [K][2][H][W].
int oracle_tv_shrink(int H, int W, int K, const double* g, double t, int per_label, double* v) {
  if (H < 1 || W < 1 || K < 1 || t < 0.0) return -1;
  tv_shrink(H, W, K, g, t, per_label, v);
  return 0;
}

// T iterations of the ADMM for the TV model, in place (v, bv: [K][2][H][W];
// w, bw, u: [K][H][W]):
//   u   = (I + grad^T grad)^(-1) [ grad^T (v - b_v) + (w - b_w) - gamma s ]
//   g_v = b_v + grad u ;  v = vector shrinkage of g_v by gamma lambda
//   g_w = b_w + u      ;  w = P_C(g_w) pixelwise
//   b_v = g_v - v      ;  b_w = g_w - w
// fp_res (nullable, length T): the fixed-point residual of each iteration, as
// in oracle_admm_iterate.
int oracle_tv_admm_iterate(int H, int W, int K, const double* s, double lambda, double gamma, int per_label, int T,
                           double* v, double* bv, double* w, double* bw, double* u, double* fp_res) {
  if (H < 2 || W < 2 || K < 1 || T < 0 || !(gamma > 0.0) || lambda < 0.0) return -1;
  const size_t P = static_cast<size_t>(H) * W, KP = static_cast<size_t>(K) * P, NV = 2 * KP;
  const double t = gamma * lambda;
  std::vector<double> diff(NV), rhs(KP), gu(NV), vn(NV), gw(K), x(K);
  for (int it = 0; it < T; ++it) {
    for (size_t i = 0; i < NV; ++i) diff[i] = v[i] - bv[i];
    for (int k = 0; k < K; ++k) tv_grad_adj(H, W, diff.data() + 2 * k * P, rhs.data() + k * P);
    for (size_t i = 0; i < KP; ++i) rhs[i] += (w[i] - bw[i]) - gamma * s[i];
    parallel_for(K, [&](int k) { tv_solve_one(H, W, rhs.data() + k * P, u + k * P); });
    for (int k = 0; k < K; ++k) tv_grad(H, W, u + k * P, gu.data() + 2 * k * P);
    for (size_t i = 0; i < NV; ++i) gu[i] += bv[i];  // g_v
    tv_shrink(H, W, K, gu.data(), t, per_label, vn.data());
    double res = 0.0;
    for (size_t i = 0; i < NV; ++i) {
      const double bn = gu[i] - vn[i];
      res += (vn[i] - v[i]) * (vn[i] - v[i]) + (bn - bv[i]) * (bn - bv[i]);
      v[i] = vn[i];
      bv[i] = bn;
    }
    for (size_t r = 0; r < P; ++r) {
      for (int k = 0; k < K; ++k) gw[k] = bw[k * P + r] + u[k * P + r];
      project_simplex_sort(gw.data(), K, x.data());
      for (int k = 0; k < K; ++k) {
        const double bn = gw[k] - x[k];
        res += (x[k] - w[k * P + r]) * (x[k] - w[k * P + r]) + (bn - bw[k * P + r]) * (bn - bw[k * P + r]);
        w[k * P + r] = x[k];
        bw[k * P + r] = bn;
      }
    }
    if (fp_res) fp_res[it] = res;
  }
  return 0;
}

// Energy of the TV model at x: <x, s> + lambda sum_pixels |(I_q (x) grad) x|.
int oracle_tv_energy(int H, int W, int K, const double* x, const double* s, double lambda, int per_label,
                     double* energy) {
  if (H < 2 || W < 2 || K < 1) return -1;
  const size_t P = static_cast<size_t>(H) * W;
  std::vector<double> g(2 * K * P);
  for (int k = 0; k < K; ++k) tv_grad(H, W, x + k * P, g.data() + 2 * k * P);
  double data = 0.0, reg = 0.0;
  for (size_t i = 0; i < static_cast<size_t>(K) * P; ++i) data += x[i] * s[i];
  for (size_t r = 0; r < P; ++r) {
    if (per_label) {
      for (int k = 0; k < K; ++k)
        reg += std::sqrt(g[2 * k * P + r] * g[2 * k * P + r] + g[(2 * k + 1) * P + r] * g[(2 * k + 1) * P + r]);
    } else {
      double n2 = 0.0;
      for (int i = 0; i < 2 * K; ++i) n2 += g[i * P + r] * g[i * P + r];
      reg += std::sqrt(n2);
    }
  }
  *energy = data + lambda * reg;
  return 0;
}

}  // extern "C"

// ===========================================================================
// NL-means regulariser, the second comparison model of Sec. 4: the gradient
// of the TV model replaced by a matrix D built from patch similarities of f.
//   * patch distance d_a(i, j) = sum_{|t1|,|t2| <= h} G_a(t) sum_ch
//     (f(i + t) - f(j + t))^2, h = ceil((p - 1)/2), G_a the Gaussian of
//     standard deviation a on the patch, normalised to sum 1;
//   * pixels i in raster order pick k = min(mt, 2 mt - l) new neighbours j
//     (l: i's neighbours so far) among the candidates of the varpi x varpi
//     search window with the smallest d_a(i, j), and set w(i, j) = w(j, i) = 1;
//   * D has m = 2 mt blocks; block b, row i: -1 at i and +1 at i's b-th
//     neighbour (a zero row when i has fewer than b + 1 neighbours).
// Readings (the paper leaves them open): the window is clipped to the image
// and f is mirrored at the border for the patches (index -1 -> 1); the
// distance is taken over all channels; candidates are ordered by (distance,
// raster index); a candidate already linked to i, or whose neighbour count
// has reached 2 mt, is passed over (so that no row needs more than m
// blocks); neighbours are listed in increasing raster index.  The regulariser
// is the isotropic one, lambda sum_i (sum_k sum_b ((D u_k)_b(i))^2)^(1/2);
// the ADMM is that of Sec. 3 with S replaced by D, whose u-step solves
// (I + D^T D) u = rhs (here by conjugate gradients to a relative residual of
// 1e-13: the exact solve).  The distances are summed in a fixed order
// without fused multiply-adds, so that the integer graph does not depend on
// the compiler.
// ===========================================================================
namespace {

int mirror(int x, int n) {
  while (x < 0 || x >= n) x = x < 0 ? -x : 2 * (n - 1) - x;
  return x;
}

std::vector<double> nl_patch_weights(int p, double a) {
  const int h = p / 2;  // ceil((p - 1)/2) for integer p
  const int n = 2 * h + 1;
  std::vector<double> G(static_cast<size_t>(n) * n);
  double sum = 0.0;
  for (int t1 = -h; t1 <= h; ++t1)
    for (int t2 = -h; t2 <= h; ++t2) {
      const double g = std::exp(-static_cast<double>(t1 * t1 + t2 * t2) / (2.0 * a * a));
      G[(t1 + h) * n + (t2 + h)] = g;
      sum += g;
    }
  for (double& g : G) g /= sum;
  return G;
}

double nl_dist(int H, int W, int C, const double* f, const std::vector<double>& G, int h, int ri, int ci, int rj,
               int cj) {
  const size_t P = static_cast<size_t>(H) * W;
  const int n = 2 * h + 1;
  double acc = 0.0;
  for (int t1 = -h; t1 <= h; ++t1)
    for (int t2 = -h; t2 <= h; ++t2) {
      const size_t a = static_cast<size_t>(mirror(ri + t1, H)) * W + mirror(ci + t2, W);
      const size_t b = static_cast<size_t>(mirror(rj + t1, H)) * W + mirror(cj + t2, W);
      double s = 0.0;
      for (int ch = 0; ch < C; ++ch) {
        const double d = f[ch * P + a] - f[ch * P + b];
        const double dd = d * d;
        s = s + dd;
      }
      const double term = G[(t1 + h) * n + (t2 + h)] * s;
      acc = acc + term;
    }
  return acc;
}

// Neighbour lists nbr[i][0 .. m) (increasing index, -1 padded) and counts.
void nl_graph(int H, int W, int C, const double* f, int p, int win, double a, int mt, std::vector<int>& nbr,
              std::vector<int>& deg) {
  const size_t P = static_cast<size_t>(H) * W;
  const int m = 2 * mt, r = win / 2, h = p / 2;
  const auto G = nl_patch_weights(p, a);
  std::vector<std::vector<int>> lists(P);
  deg.assign(P, 0);
  std::vector<std::pair<double, int>> cand;
  for (int ri = 0; ri < H; ++ri)
    for (int ci = 0; ci < W; ++ci) {
      const int i = ri * W + ci;
      cand.clear();
      for (int rj = std::max(0, ri - r); rj <= std::min(H - 1, ri + r); ++rj)
        for (int cj = std::max(0, ci - r); cj <= std::min(W - 1, ci + r); ++cj) {
          const int j = rj * W + cj;
          if (j != i) cand.push_back({nl_dist(H, W, C, f, G, h, ri, ci, rj, cj), j});
        }
      std::sort(cand.begin(), cand.end());
      const int k = std::min(mt, m - deg[i]);
      int taken = 0;
      for (const auto& c : cand) {
        if (taken >= k) break;
        const int j = c.second;
        if (deg[j] >= m) continue;
        if (std::find(lists[i].begin(), lists[i].end(), j) != lists[i].end()) continue;
        lists[i].push_back(j);
        lists[j].push_back(i);
        ++deg[i];
        ++deg[j];
        ++taken;
      }
    }
  nbr.assign(P * m, -1);
  for (size_t i = 0; i < P; ++i) {
    std::sort(lists[i].begin(), lists[i].end());
    for (size_t b = 0; b < lists[i].size(); ++b) nbr[i * m + b] = lists[i][b];
  }
}

// (D x)_b(i) = x(nbr_b(i)) - x(i) for one plane: out [m][P].
void nl_D(size_t P, int m, const int* nbr, const double* x, double* out) {
  for (int b = 0; b < m; ++b)
    for (size_t i = 0; i < P; ++i) {
      const int j = nbr[i * m + b];
      out[b * P + i] = j >= 0 ? x[j] - x[i] : 0.0;
    }
}

// D^T q for one plane, by scattering the rows of D: q [m][P] -> out [P].
void nl_Dt(size_t P, int m, const int* nbr, const double* q, double* out) {
  std::fill(out, out + P, 0.0);
  for (size_t i = 0; i < P; ++i)
    for (int b = 0; b < m; ++b) {
      const int j = nbr[i * m + b];
      if (j < 0) continue;
      out[j] += q[b * P + i];
      out[i] -= q[b * P + i];
    }
}

// (I + D^T D) x for one plane.
void nl_apply(size_t P, int m, const int* nbr, const double* x, double* y, std::vector<double>& tmp) {
  tmp.resize(static_cast<size_t>(m) * P);
  nl_D(P, m, nbr, x, tmp.data());
  nl_Dt(P, m, nbr, tmp.data(), y);
  for (size_t i = 0; i < P; ++i) y[i] += x[i];
}

// Conjugate gradients for (I + D^T D) u = rhs from u = 0 until the residual
// is below 1e-13 of |rhs| (I + D^T D is symmetric positive definite with
// eigenvalues in [1, 1 + 4 m]).
void nl_solve_one(size_t P, int m, const int* nbr, const double* rhs, double* u) {
  std::vector<double> r(rhs, rhs + P), d(rhs, rhs + P), q(P), tmp;
  std::fill(u, u + P, 0.0);
  double rr = 0.0;
  for (size_t i = 0; i < P; ++i) rr += r[i] * r[i];
  const double stop = 1e-26 * std::max(rr, 1e-300);
  for (int it = 0; it < 2000 && rr > stop; ++it) {
    nl_apply(P, m, nbr, d.data(), q.data(), tmp);
    double dq = 0.0;
    for (size_t i = 0; i < P; ++i) dq += d[i] * q[i];
    const double alpha = rr / dq;
    double rr2 = 0.0;
    for (size_t i = 0; i < P; ++i) {
      u[i] += alpha * d[i];
      r[i] -= alpha * q[i];
      rr2 += r[i] * r[i];
    }
    const double beta = rr2 / rr;
    for (size_t i = 0; i < P; ++i) d[i] = r[i] + beta * d[i];
    rr = rr2;
  }
}

}  // namespace

extern "C" {

// Patch distance d_a(i, j) between pixels (ri, ci) and (rj, cj) of f [C][H][W].
double oracle_nl_distance(int H, int W, int C, const double* f, int p, double a, int ri, int ci, int rj, int cj) {
  const auto G = nl_patch_weights(p, a);
  return nl_dist(H, W, C, f, G, p / 2, ri, ci, rj, cj);
}

// The neighbour graph of f [C][H][W]: nbr [H W][2 mt] (increasing index, -1
// padded) and deg [H W].
int oracle_nl_graph(int H, int W, int C, const double* f, int p, int win, double a, int mt, int* nbr, int* deg) {
  if (H < 2 || W < 2 || C < 1 || p < 1 || win < 3 || !(a > 0.0) || mt < 1) return -1;
  std::vector<int> n, d;
  nl_graph(H, W, C, f, p, win, a, mt, n, d);
  std::copy(n.begin(), n.end(), nbr);
  std::copy(d.begin(), d.end(), deg);
  return 0;
}

// D and D^T for K planes: u [K][H][W] <-> q [K][m][H][W].
int oracle_nl_D(int H, int W, int K, int m, const int* nbr, const double* u, double* q) {
  const size_t P = static_cast<size_t>(H) * W;
  for (int k = 0; k < K; ++k) nl_D(P, m, nbr, u + k * P, q + static_cast<size_t>(k) * m * P);
  return 0;
}

int oracle_nl_Dt(int H, int W, int K, int m, const int* nbr, const double* q, double* u) {
  const size_t P = static_cast<size_t>(H) * W;
  for (int k = 0; k < K; ++k) nl_Dt(P, m, nbr, q + static_cast<size_t>(k) * m * P, u + k * P);
  return 0;
}

// (I + D^T D)^(-1) rhs for K planes.
int oracle_nl_solve(int H, int W, int K, int m, const int* nbr, const double* rhs, double* u) {
  const size_t P = static_cast<size_t>(H) * W;
  parallel_for(K, [&](int k) { nl_solve_one(P, m, nbr, rhs + k * P, u + k * P); });
  return 0;
}

// T iterations of the ADMM for the NL model, in place (v, bv [K][m][H][W];
// w, bw, u [K][H][W]), the TV iteration with grad replaced by D; the group of
// the shrinkage is all m K values of a pixel.
int oracle_nl_admm_iterate(int H, int W, int K, int m, const int* nbr, const double* s, double lambda, double gamma,
                           int T, double* v, double* bv, double* w, double* bw, double* u, double* fp_res) {
  if (H < 2 || W < 2 || K < 1 || m < 1 || T < 0 || !(gamma > 0.0) || lambda < 0.0) return -1;
  const size_t P = static_cast<size_t>(H) * W, KP = static_cast<size_t>(K) * P, NV = static_cast<size_t>(m) * KP;
  const double t = gamma * lambda;
  std::vector<double> diff(NV), rhs(KP), g(NV), vn(NV), gw(K), x(K);
  for (int it = 0; it < T; ++it) {
    for (size_t i = 0; i < NV; ++i) diff[i] = v[i] - bv[i];
    for (int k = 0; k < K; ++k) nl_Dt(P, m, nbr, diff.data() + k * m * P, rhs.data() + k * P);
    for (size_t i = 0; i < KP; ++i) rhs[i] += (w[i] - bw[i]) - gamma * s[i];
    parallel_for(K, [&](int k) { nl_solve_one(P, m, nbr, rhs.data() + k * P, u + k * P); });
    for (int k = 0; k < K; ++k) nl_D(P, m, nbr, u + k * P, g.data() + k * m * P);
    for (size_t i = 0; i < NV; ++i) g[i] += bv[i];
    for (size_t px = 0; px < P; ++px) shrink_group(g.data() + px, m * K, P, t, vn.data() + px);
    double res = 0.0;
    for (size_t i = 0; i < NV; ++i) {
      const double bn = g[i] - vn[i];
      res += (vn[i] - v[i]) * (vn[i] - v[i]) + (bn - bv[i]) * (bn - bv[i]);
      v[i] = vn[i];
      bv[i] = bn;
    }
    for (size_t px = 0; px < P; ++px) {
      for (int k = 0; k < K; ++k) gw[k] = bw[k * P + px] + u[k * P + px];
      project_simplex_sort(gw.data(), K, x.data());
      for (int k = 0; k < K; ++k) {
        const double bn = gw[k] - x[k];
        res += (x[k] - w[k * P + px]) * (x[k] - w[k * P + px]) + (bn - bw[k * P + px]) * (bn - bw[k * P + px]);
        w[k * P + px] = x[k];
        bw[k * P + px] = bn;
      }
    }
    if (fp_res) fp_res[it] = res;
  }
  return 0;
}

// Energy of the NL model at x: <x, s> + lambda sum_i |(I_q (x) D) x|(i).
int oracle_nl_energy(int H, int W, int K, int m, const int* nbr, const double* x, const double* s, double lambda,
                     double* energy) {
  const size_t P = static_cast<size_t>(H) * W;
  std::vector<double> q(static_cast<size_t>(K) * m * P);
  for (int k = 0; k < K; ++k) nl_D(P, m, nbr, x + k * P, q.data() + k * m * P);
  double data = 0.0, reg = 0.0;
  for (size_t i = 0; i < static_cast<size_t>(K) * P; ++i) data += x[i] * s[i];
  for (size_t px = 0; px < P; ++px) {
    double n2 = 0.0;
    for (size_t c = 0; c < static_cast<size_t>(K) * m; ++c) n2 += q[c * P + px] * q[c * P + px];
    reg += std::sqrt(n2);
  }
  *energy = data + lambda * reg;
  return 0;
}

}  // extern "C"

// Host-side check of the radix-16 row FFT building blocks (shf_fft16.cuh)
// against FP64 DFTs, for the half widths 64, 128, 256, 512 and 1024, and the
// two-rows-per-transform packing for widths 128, 256 and 512, and the column
// (batch) layout for heights 512, 1024 (8 columns) and 2048 (4 columns).  A row group
// of T threads is emulated lane by lane, phase by phase, exactly as the kernel
// sequences them between warp barriers: butterflies, Stockham stores to the
// padded group buffer, stride reads, and the packing steps with each lane's
// partner values taken from a snapshot of the registers before the step (what
// a warp shuffle returns).  Prints one line per length and exits non-zero on
// a failed bound.
#include <array>
#include <cmath>
#include <complex>
#include <cstdio>
#include <random>
#include <vector>

#include "shf_fft16.cuh"

using namespace shf;
using cd = std::complex<double>;
using Regs = std::array<float2, 16>;

static float2 (&regs(Regs& r))[16] { return *reinterpret_cast<float2(*)[16]>(r.data()); }

template <int N, int P, int S>
static void bfly_all(std::vector<Regs>& V, const float2* pt) {
  for (int tt = 0; tt < N / 16; ++tt) r16::pass_bfly<N, P, S>(regs(V[tt]), tt, pt);
}

// The whole transform of one row group (r16::row_fft's sequence of phases).
template <int N, int S>
static void group_fft(std::vector<Regs>& V, std::vector<float2>& buf, const float2* pt) {
  using PS = r16::Passes<N>;
  constexpr int T = PS::T;
  bfly_all<N, 0, S>(V, pt);
  if constexpr (PS::NPASS > 1) {
    for (int tt = 0; tt < T; ++tt) r16::pass_store<N, 0>(regs(V[tt]), tt, buf.data());
    for (int tt = 0; tt < T; ++tt) r16::load_stride<N>(regs(V[tt]), tt, buf.data());
    bfly_all<N, (PS::NPASS > 1 ? 1 : 0), S>(V, pt);
  }
  if constexpr (PS::NPASS > 2) {
    for (int tt = 0; tt < T; ++tt) r16::pass_store<N, (PS::NPASS > 2 ? 1 : 0)>(regs(V[tt]), tt, buf.data());
    for (int tt = 0; tt < T; ++tt) r16::load_stride<N>(regs(V[tt]), tt, buf.data());
    bfly_all<N, (PS::NPASS > 2 ? 2 : 0), S>(V, pt);
  }
}

template <int L>
static int check() {
  using PS = r16::Passes<L>;
  constexpr int T = PS::T;
  const int W = 2 * L;
  std::vector<float2> tw(W);  // exp(-2 pi i m / W), as the library's table
  for (int m = 0; m < W; ++m) tw[m] = make_float2(std::cos(-2 * M_PI * m / W), std::sin(-2 * M_PI * m / W));
  std::vector<float2> pt(PS::TWSIZE);
  r16::build_pass_twiddles<L, 2>(pt.data(), tw.data(), 0, 1);
  std::vector<float2> buf(reg::row_buf(L), make_float2(NAN, NAN));
  std::mt19937 rng(1805 + L);
  std::normal_distribution<double> nd;
  auto partner = [](int tt) { return (T - tt) & (T - 1); };

  // 1. complex transform, both exponent signs
  double e_fft = 0;
  for (int S : {+1, -1}) {
    std::vector<cd> x(L);
    for (auto& a : x) a = cd(nd(rng), nd(rng));
    std::vector<Regs> V(T);
    for (int tt = 0; tt < T; ++tt)
      for (int k = 0; k < 16; ++k) V[tt][k] = make_float2(x[tt + k * T].real(), x[tt + k * T].imag());
    if (S > 0)
      group_fft<L, +1>(V, buf, pt.data());
    else
      group_fft<L, -1>(V, buf, pt.data());
    for (int q = 0; q < L; ++q) {
      cd ref = 0;
      for (int n = 0; n < L; ++n) ref += x[n] * std::polar(1.0, S * 2 * M_PI * double(n) * q / L);
      const float2 g = V[q % T][q / T];
      e_fft = std::max(e_fft, std::abs(cd(g.x, g.y) - ref) / std::sqrt(double(L)));
    }
  }

  // 2. real row: X = rfft(x); packing + inverse gives W (x[2n] + i x[2n+1]);
  //    forward + unpacking gives X back
  std::vector<double> xr(W);
  for (auto& a : xr) a = nd(rng);
  std::vector<cd> X(L + 1);
  for (int k = 0; k <= L; ++k) {
    cd s = 0;
    for (int m = 0; m < W; ++m) s += xr[m] * std::polar(1.0, -2 * M_PI * double(k) * m / W);
    X[k] = s;
  }
  auto f2 = [](cd a) { return make_float2(float(a.real()), float(a.imag())); };
  std::vector<Regs> V(T);
  for (int tt = 0; tt < T; ++tt)
    for (int k = 0; k < 16; ++k) V[tt][k] = f2(X[tt + k * T]);
  std::vector<float2> prev(T, f2(X[L]));
  for (int k = 0; k < 8; ++k) {
    const std::vector<Regs> snap = V;
    for (int tt = 0; tt < T; ++tt) {
      const Regs& p = snap[partner(tt)];
      r16::pack_step<L>(regs(V[tt]), k, tt, p[15 - k], p[k], prev[tt], tw.data());
    }
  }
  group_fft<L, +1>(V, buf, pt.data());
  double e_inv = 0;
  for (int n = 0; n < L; ++n) {
    const float2 g = V[n % T][n / T];
    e_inv = std::max(e_inv, std::abs(cd(g.x, g.y) / double(W) - cd(xr[2 * n], xr[2 * n + 1])));
  }
  for (auto& r : V)
    for (auto& a : r) a = c_scale(a, 1.f / W);
  group_fft<L, -1>(V, buf, pt.data());
  double e_fwd = 0, xmax = 0;
  for (int tt = 0; tt < T; ++tt)
    for (int q = 0; q < 16; ++q) {
      const float2 o = r16::unpack_value<L>(regs(V[tt]), q, tt, V[partner(tt)][15 - q], tw.data());
      e_fwd = std::max(e_fwd, std::abs(cd(o.x, o.y) - X[tt + q * T]));
    }
  e_fwd = std::max(e_fwd, std::abs(cd(V[0][0].x - V[0][0].y, 0.0) - X[L]));
  for (const auto& a : X) xmax = std::max(xmax, std::abs(a));

  // FP32 transforms: error ~ eps log2(L) times the data scale; bounds with a
  // margin of about 10
  const double eps = 6e-8, lg = std::log2(double(L));
  const bool ok = e_fft < 10 * eps * lg * 4 && e_inv < 10 * eps * lg * 4 && e_fwd < 10 * eps * lg * xmax;
  std::printf("L=%d T=%d passes=%d fft %.2e inverse-real %.2e forward-real %.2e (|X| <= %.1f) %s\n", L, T,
              PS::NPASS, e_fft, e_inv, e_fwd, xmax, ok ? "ok" : "FAIL");
  return ok ? 0 : 1;
}

// Two real rows as one complex row of length W (r16::pair_pack / pair_unpack):
// packing + inverse gives W (a + i b); forward + unpacking gives both half
// spectra back.
template <int W>
static int check_pair() {
  using PS = r16::Passes<W>;
  constexpr int T = PS::T, L = W / 2;
  std::vector<float2> tw(W);
  for (int m = 0; m < W; ++m) tw[m] = make_float2(std::cos(-2 * M_PI * m / W), std::sin(-2 * M_PI * m / W));
  std::vector<float2> pt(PS::TWSIZE);
  r16::build_pass_twiddles<W, 1>(pt.data(), tw.data(), 0, 1);
  std::vector<float2> buf(reg::row_buf(W), make_float2(NAN, NAN));
  std::mt19937 rng(2 * W + 1);
  std::normal_distribution<double> nd;
  std::vector<double> a(W), b(W);
  for (int m = 0; m < W; ++m) a[m] = nd(rng), b[m] = nd(rng);
  std::vector<cd> Xa(L + 1), Xb(L + 1);
  for (int k = 0; k <= L; ++k) {
    cd sa = 0, sb = 0;
    for (int m = 0; m < W; ++m) {
      const cd e = std::polar(1.0, -2 * M_PI * double(k) * m / W);
      sa += a[m] * e;
      sb += b[m] * e;
    }
    Xa[k] = sa, Xb[k] = sb;
  }
  auto f2 = [](cd z) { return make_float2(float(z.real()), float(z.imag())); };
  std::vector<Regs> V(T);
  for (int tt = 0; tt < T; ++tt)
    for (int k = 0; k < 16; ++k) {
      const int n = tt + k * T;
      const bool up = n > L;
      const int m = up ? W - n : n;
      V[tt][k] = r16::pair_pack(f2(Xa[m]), f2(Xb[m]), up);
    }
  group_fft<W, +1>(V, buf, pt.data());
  double e_inv = 0;
  for (int m = 0; m < W; ++m) {
    const float2 g = V[m % T][m / T];
    e_inv = std::max(e_inv, std::abs(cd(g.x, g.y) / double(W) - cd(a[m], b[m])));
  }
  for (auto& r : V)
    for (auto& z : r) z = c_scale(z, 1.f / W);
  group_fft<W, -1>(V, buf, pt.data());
  double e_fwd = 0, xmax = 0;
  for (int tt = 0; tt < T; ++tt)
    for (int q = 0; q <= 8; ++q) {
      const int k = tt + q * T;
      if (k > L) continue;
      const float2 dm = r16::pair_partner(tt, V[(T - tt) & (T - 1)][15 - q], V[tt][(16 - q) & 15]);
      float2 xa, xb;
      r16::pair_unpack(V[tt][q], dm, xa, xb);
      e_fwd = std::max(e_fwd, std::max(std::abs(cd(xa.x, xa.y) - Xa[k]), std::abs(cd(xb.x, xb.y) - Xb[k])));
    }
  for (int k = 0; k <= L; ++k) xmax = std::max(xmax, std::max(std::abs(Xa[k]), std::abs(Xb[k])));
  const double eps = 6e-8, lg = std::log2(double(W));
  const bool ok = e_inv < 10 * eps * lg * 4 && e_fwd < 10 * eps * lg * xmax;
  std::printf("pair W=%d T=%d inverse %.2e forward %.2e (|X| <= %.1f) %s\n", W, T, e_inv, e_fwd, xmax,
              ok ? "ok" : "FAIL");
  return ok ? 0 : 1;
}

// The column (batch) layout of r16::batch_fft: KB columns, element i of
// column b at ridx(i) KB + b, thread (b, tt); checked against FP64 DFTs.
template <int N, int KB>
static int check_batch() {
  using PS = r16::Passes<N>;
  constexpr int T = PS::T;
  std::vector<float2> tw(N);
  for (int m = 0; m < N; ++m) tw[m] = make_float2(std::cos(-2 * M_PI * m / N), std::sin(-2 * M_PI * m / N));
  std::vector<float2> pt(PS::TWSIZE);
  r16::build_pass_twiddles<N, 1>(pt.data(), tw.data(), 0, 1);
  std::vector<float2> buf0(r16::brows16(N) * KB, make_float2(NAN, NAN)), buf1 = buf0;
  std::mt19937 rng(3 * N + KB);
  std::normal_distribution<double> nd;
  std::vector<std::vector<cd>> x(KB, std::vector<cd>(N));
  for (auto& c : x)
    for (auto& a : c) a = cd(nd(rng), nd(rng));
  std::vector<Regs> V(T * KB);  // thread (b, tt) at tt * KB + b
  for (int tt = 0; tt < T; ++tt)
    for (int b = 0; b < KB; ++b)
      for (int k = 0; k < 16; ++k) V[tt * KB + b][k] = make_float2(x[b][tt + k * T].real(), x[b][tt + k * T].imag());
  // the phases of batch_fft<N, +1, KB> with every thread of the CTA in turn
  auto bfly = [&](auto P) {
    for (int t = 0; t < T * KB; ++t) r16::pass_bfly<N, decltype(P)::value, +1>(regs(V[t]), t / KB, pt.data());
  };
  bfly(std::integral_constant<int, 0>());
  if constexpr (PS::NPASS > 1) {
    for (int t = 0; t < T * KB; ++t) r16::bpass_store<N, 0, KB>(regs(V[t]), t / KB, t % KB, buf0.data());
    for (int t = 0; t < T * KB; ++t) r16::bload_stride<N, KB>(regs(V[t]), t / KB, t % KB, buf0.data());
    bfly(std::integral_constant<int, (PS::NPASS > 1 ? 1 : 0)>());
  }
  if constexpr (PS::NPASS > 2) {
    for (int t = 0; t < T * KB; ++t)
      r16::bpass_store<N, (PS::NPASS > 2 ? 1 : 0), KB>(regs(V[t]), t / KB, t % KB, buf1.data());
    for (int t = 0; t < T * KB; ++t) r16::bload_stride<N, KB>(regs(V[t]), t / KB, t % KB, buf1.data());
    bfly(std::integral_constant<int, (PS::NPASS > 2 ? 2 : 0)>());
  }
  double e = 0;
  for (int b = 0; b < KB; ++b)
    for (int q = 0; q < N; ++q) {
      cd ref = 0;
      for (int n = 0; n < N; ++n) ref += x[b][n] * std::polar(1.0, 2 * M_PI * double(n) * q / N);
      const float2 g = V[(q % T) * KB + b][q / T];
      e = std::max(e, std::abs(cd(g.x, g.y) - ref) / std::sqrt(double(N)));
    }
  const bool ok = e < 10 * 6e-8 * std::log2(double(N)) * 4;
  std::printf("batch N=%d KB=%d err %.2e %s\n", N, KB, e, ok ? "ok" : "FAIL");
  return ok ? 0 : 1;
}

int main() {
  return check<64>() + check<128>() + check<256>() + check<512>() + check<1024>() + check_pair<128>() +
         check_pair<256>() + check_pair<512>() + check_batch<512, 8>() + check_batch<1024, 8>() +
         check_batch<2048, 4>();
}

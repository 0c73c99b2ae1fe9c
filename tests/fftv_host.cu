// Host-side check of the V-value FFT building blocks (shf_fftv.cuh) against
// FP64 DFTs: rows for the half widths 3 2^a (V = 12), 5 2^a (V = 20) and 1024
// (V = 32) with row groups of 2 to 32 threads, and column batches.  A row
// group of T threads is emulated lane by lane, phase by phase, exactly as the
// kernel sequences them between warp barriers: butterflies, Stockham stores
// to the group buffer, stride reads, and the packing steps with each lane's
// partner values taken from a snapshot of the registers before the step (what
// a warp shuffle returns).  Prints one line per length and exits non-zero on
// a failed bound.
#include <array>
#include <cmath>
#include <complex>
#include <cstdio>
#include <random>
#include <vector>

#include "shf_fftv.cuh"

using namespace shf;
using cd = std::complex<double>;

template <int L>
struct Emu {
  using PS = rv::Passes<L>;
  static constexpr int V = PS::V, T = PS::T;
  using Regs = std::array<float2, V>;
  static float2 (&regs(Regs& r))[V] { return *reinterpret_cast<float2(*)[V]>(r.data()); }

  template <int P, int S>
  static void bfly_all(std::vector<Regs>& R, const float2* pt) {
    for (int tt = 0; tt < T; ++tt) rv::pass_bfly<L, P, S>(regs(R[tt]), tt, pt);
  }
  // rv::row_fft's sequence of phases over the whole group
  template <int S, int P = 0>
  static void group_fft(std::vector<Regs>& R, std::vector<float2>& buf, const float2* pt) {
    bfly_all<P, S>(R, pt);
    if constexpr (P + 1 < PS::NPASS) {
      for (int tt = 0; tt < T; ++tt) rv::pass_store<L, P>(regs(R[tt]), tt, buf.data());
      for (int tt = 0; tt < T; ++tt) rv::load_stride<L, P>(regs(R[tt]), tt, buf.data());
      group_fft<S, P + 1>(R, buf, pt);
    }
  }

  // the exchange layout after pass P: inside the buffer and one slot per index
  template <int P = 0>
  static bool layout_ok() {
    if constexpr (P + 1 < PS::NPASS) {
      std::vector<int> seen(rv::row_buf(L), 0);
      for (int i = 0; i < L; ++i) {
        const int a = rv::xidx<L, P>(i);
        if (a < 0 || a >= rv::row_buf(L) || seen[a]++) return false;
      }
      return layout_ok<P + 1>();
    }
    return true;
  }

  static int check() {
    if (!layout_ok()) {
      std::printf("L=%d exchange layout out of the buffer or not injective FAIL\n", L);
      return 1;
    }
    const int W = 2 * L;
    std::vector<float2> tw(W);  // exp(-2 pi i m / W), as the library's table
    for (int m = 0; m < W; ++m) tw[m] = make_float2(std::cos(-2 * M_PI * m / W), std::sin(-2 * M_PI * m / W));
    std::vector<float2> pt(PS::TWSIZE);
    rv::build_pass_twiddles<L, 2>(pt.data(), tw.data(), 0, 1);
    std::vector<float2> buf(rv::row_buf(L), make_float2(NAN, NAN));
    std::mt19937 rng(1805 + L);
    std::normal_distribution<double> nd;
    auto partner = [](int tt) { return (T - tt) & (T - 1); };

    // 1. complex transform, both exponent signs
    double e_fft = 0;
    for (int S : {+1, -1}) {
      std::vector<cd> x(L);
      for (auto& a : x) a = cd(nd(rng), nd(rng));
      std::vector<Regs> R(T);
      for (int tt = 0; tt < T; ++tt)
        for (int k = 0; k < V; ++k) R[tt][k] = make_float2(x[tt + k * T].real(), x[tt + k * T].imag());
      if (S > 0)
        group_fft<+1>(R, buf, pt.data());
      else
        group_fft<-1>(R, buf, pt.data());
      for (int q = 0; q < L; ++q) {
        cd ref = 0;
        for (int n = 0; n < L; ++n) ref += x[n] * std::polar(1.0, S * 2 * M_PI * double(n) * q / L);
        const float2 g = R[q % T][q / T];
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
    std::vector<Regs> R(T);
    for (int tt = 0; tt < T; ++tt)
      for (int k = 0; k < V; ++k) R[tt][k] = f2(X[tt + k * T]);
    std::vector<float2> prev(T, f2(X[L]));
    for (int k = 0; k < V / 2; ++k) {
      const std::vector<Regs> snap = R;
      for (int tt = 0; tt < T; ++tt) {
        const Regs& p = snap[partner(tt)];
        rv::pack_step<L>(regs(R[tt]), k, tt, p[V - 1 - k], p[k], prev[tt], tw.data());
      }
    }
    group_fft<+1>(R, buf, pt.data());
    double e_inv = 0;
    for (int n = 0; n < L; ++n) {
      const float2 g = R[n % T][n / T];
      e_inv = std::max(e_inv, std::abs(cd(g.x, g.y) / double(W) - cd(xr[2 * n], xr[2 * n + 1])));
    }
    for (auto& r : R)
      for (auto& a : r) a = c_scale(a, 1.f / W);
    group_fft<-1>(R, buf, pt.data());
    double e_fwd = 0, xmax = 0;
    for (int tt = 0; tt < T; ++tt)
      for (int q = 0; q < V; ++q) {
        const float2 o = rv::unpack_value<L>(regs(R[tt]), q, tt, R[partner(tt)][V - 1 - q], tw.data());
        e_fwd = std::max(e_fwd, std::abs(cd(o.x, o.y) - X[tt + q * T]));
      }
    e_fwd = std::max(e_fwd, std::abs(cd(R[0][0].x - R[0][0].y, 0.0) - X[L]));
    for (const auto& a : X) xmax = std::max(xmax, std::abs(a));

    // FP32 transforms: error ~ eps log2(L) times the data scale; bounds with a
    // margin of about 10
    const double eps = 6e-8, lg = std::log2(double(L));
    const bool ok = e_fft < 10 * eps * lg * 4 && e_inv < 10 * eps * lg * 4 && e_fwd < 10 * eps * lg * xmax;
    std::printf("L=%d V=%d T=%d passes=%d fft %.2e inverse-real %.2e forward-real %.2e (|X| <= %.1f) %s\n", L, V,
                T, PS::NPASS, e_fft, e_inv, e_fwd, xmax, ok ? "ok" : "FAIL");
    return ok ? 0 : 1;
  }
};

// rv::batch_fft over KB columns of length N (threads (b, tt), alternating
// exchange buffers of brows(N) KB elements), against FP64 DFTs per column.
template <int N, int KB>
struct BatchEmu {
  using PS = rv::Passes<N>;
  static constexpr int V = PS::V, T = PS::T, BR = rv::brows(N) * KB;
  using Regs = std::array<float2, V>;
  static float2 (&regs(Regs& r))[V] { return *reinterpret_cast<float2(*)[V]>(r.data()); }

  template <int P = 0>
  static bool layout_ok() {
    if constexpr (P + 1 < PS::NPASS) {
      std::vector<int> seen(BR, 0);
      for (int i = 0; i < N; ++i)
        for (int b = 0; b < KB; ++b) {
          const int a = rv::bxidx<N, P, KB>(i) * KB + b;
          if (a < 0 || a >= BR || seen[a]++) return false;
        }
      return layout_ok<P + 1>();
    }
    return true;
  }
  template <int S, int P = 0>
  static void fft(std::vector<Regs>& R, std::vector<float2>& b0, std::vector<float2>& b1, const float2* pt) {
    for (int t = 0; t < T * KB; ++t) rv::pass_bfly<N, P, S>(regs(R[t]), t / KB, pt);
    if constexpr (P + 1 < PS::NPASS) {
      std::vector<float2>& buf = (P % 2 == 0) ? b0 : b1;
      for (int t = 0; t < T * KB; ++t) rv::bpass_store<N, P, KB>(regs(R[t]), t / KB, t % KB, buf.data());
      for (int t = 0; t < T * KB; ++t) rv::bload_stride<N, P, KB>(regs(R[t]), t / KB, t % KB, buf.data());
      fft<S, P + 1>(R, b0, b1, pt);
    }
  }
  static int check() {
    if (!layout_ok()) {
      std::printf("batch N=%d KB=%d exchange layout out of the buffer or not injective FAIL\n", N, KB);
      return 1;
    }
    std::vector<float2> tw(N);  // exp(-2 pi i m / N)
    for (int m = 0; m < N; ++m) tw[m] = make_float2(std::cos(-2 * M_PI * m / N), std::sin(-2 * M_PI * m / N));
    std::vector<float2> pt(PS::TWSIZE);
    rv::build_pass_twiddles<N, 1>(pt.data(), tw.data(), 0, 1);
    std::vector<float2> b0(BR, make_float2(NAN, NAN)), b1(BR, make_float2(NAN, NAN));
    std::mt19937 rng(2011 + N + KB);
    std::normal_distribution<double> nd;
    double err = 0;
    for (int S : {+1, -1}) {
      std::vector<std::vector<cd>> x(KB, std::vector<cd>(N));
      for (auto& c : x)
        for (auto& a : c) a = cd(nd(rng), nd(rng));
      std::vector<Regs> R(T * KB);
      for (int t = 0; t < T * KB; ++t)
        for (int k = 0; k < V; ++k) {
          const cd a = x[t % KB][t / KB + k * T];
          R[t][k] = make_float2(a.real(), a.imag());
        }
      if (S > 0)
        fft<+1>(R, b0, b1, pt.data());
      else
        fft<-1>(R, b0, b1, pt.data());
      for (int b = 0; b < KB; ++b)
        for (int q = 0; q < N; ++q) {
          cd ref = 0;
          for (int n = 0; n < N; ++n) ref += x[b][n] * std::polar(1.0, S * 2 * M_PI * double(n) * q / N);
          const float2 g = R[(q % T) * KB + b][q / T];
          err = std::max(err, std::abs(cd(g.x, g.y) - ref) / std::sqrt(double(N)));
        }
    }
    const bool ok = err < 10 * 6e-8 * std::log2(double(N)) * 4;
    std::printf("batch N=%d KB=%d V=%d T=%d fft %.2e %s\n", N, KB, V, T, err, ok ? "ok" : "FAIL");
    return ok ? 0 : 1;
  }
};

int main() {
  return Emu<24>::check() + Emu<48>::check() + Emu<96>::check() + Emu<192>::check() + Emu<384>::check() +
         Emu<40>::check() + Emu<80>::check() + Emu<160>::check() + Emu<320>::check() + Emu<640>::check() +
         Emu<1024>::check() +
         BatchEmu<24, 8>::check() + BatchEmu<96, 8>::check() + BatchEmu<384, 8>::check() + BatchEmu<768, 8>::check() +
         BatchEmu<1536, 4>::check() + BatchEmu<40, 8>::check() + BatchEmu<160, 8>::check() +
         BatchEmu<640, 8>::check() + BatchEmu<1280, 4>::check() + BatchEmu<2560, 4>::check();
}

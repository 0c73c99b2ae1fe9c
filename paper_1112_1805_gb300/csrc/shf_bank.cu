// Filter bank, FFT tables and per-pixel kernels.
//
// The filter spectra follow Sec. 2 of Haeuser & Steidl (arXiv:1112.1805):
// Meyer windows v, b (Sec. 2 "Continuous Shearlets"), psi1_hat, psi2_hat
// (eq. psi1_psi2), shearlets on the cones C^h, C^v with the seam C^x and the
// scaling function varphi, discretised as in "Finite Discrete Shearlets" with
// the glued seam shearlets for |k| = 2^j.  They are evaluated in FP64 on the
// device and rounded once to FP32.
#include <cmath>
#include <cstdint>

#include "shf_internal.h"

namespace shf {

namespace {

__device__ __forceinline__ double win_v(double x) {
  if (x <= 0.0) return 0.0;
  if (x >= 1.0) return 1.0;
  return x * x * x * x * (35.0 + x * (-84.0 + x * (70.0 - 20.0 * x)));
}

__device__ __forceinline__ double win_b(double x) {
  const double a = fabs(x);
  if (a < 1.0 || a > 4.0) return 0.0;
  if (a <= 2.0) return sinpi(0.5 * win_v(a - 1.0));
  return cospi(0.5 * win_v(0.5 * a - 1.0));
}

__device__ __forceinline__ double win_psi1(double w) {
  const double p = win_b(2.0 * w), q = win_b(w);
  return sqrt(p * p + q * q);
}

__device__ __forceinline__ double win_psi2(double w) { return sqrt(win_v(w <= 0.0 ? 1.0 + w : 1.0 - w)); }

__device__ __forceinline__ double win_varphi(double w) {
  const double a = fabs(w);
  if (a <= 0.5) return 1.0;
  if (a < 1.0) return cospi(0.5 * win_v(2.0 * a - 1.0));
  return 0.0;
}

// Spectrum of one filter at integer frequency (w1, w2) of an H x W grid with
// per-axis normalised frequency xi_a = w_a 4^J / N_a.
__device__ double spectrum(FilterDesc d, long long w1, long long w2, long long H, long long W, int J) {
  if (d.kind == 0) {
    const double x1 = fabs(static_cast<double>(w1) * ldexp(1.0, 2 * J) / static_cast<double>(H));
    const double x2 = fabs(static_cast<double>(w2) * ldexp(1.0, 2 * J) / static_cast<double>(W));
    return win_varphi(fmax(x1, x2));
  }
  // |xi_1| vs |xi_2| compared exactly: |w1| W against |w2| H.
  const long long a1 = (w1 < 0 ? -w1 : w1) * W, a2 = (w2 < 0 ? -w2 : w2) * H;
  const bool cone_h = a2 < a1, cone_v = a1 < a2, seam = (a1 == a2) && a1 > 0;
  bool use_h;
  if (d.kind == 1) {
    if (!cone_h) return 0.0;
    use_h = true;
  } else if (d.kind == 2) {
    if (!cone_v) return 0.0;
    use_h = false;
  } else {  // glued: horizontal part, vertical part, seam part (horizontal formula)
    if (!(cone_h || cone_v || seam)) return 0.0;
    use_h = !cone_v;
  }
  const double scale = ldexp(1.0, 2 * (J - d.j));
  if (use_h) {
    const double x = static_cast<double>(w1) * scale / static_cast<double>(H);
    const double r = static_cast<double>(w2 * H) / static_cast<double>(w1 * W);
    return win_psi1(x) * win_psi2(ldexp(r, d.j) + static_cast<double>(d.k));
  }
  const double x = static_cast<double>(w2) * scale / static_cast<double>(W);
  const double r = static_cast<double>(w1 * W) / static_cast<double>(w2 * H);
  return win_psi1(x) * win_psi2(ldexp(r, d.j) + static_cast<double>(d.k));
}

__device__ __forceinline__ long long freq(long long n, long long N) { return n < (N + 1) / 2 ? n : n - N; }

__global__ void k_build_bank(float* __restrict__ bank, const FilterDesc* __restrict__ descs, int H, int W, int Wh,
                             int J, int eta) {
  const long long total = static_cast<long long>(eta) * H * Wh;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int n2 = static_cast<int>(e % Wh);
    const int n1 = static_cast<int>((e / Wh) % H);
    const int f = static_cast<int>(e / (static_cast<long long>(Wh) * H));
    const FilterDesc d = descs[f];
    const double a = spectrum(d, freq(n1, H), freq(n2, W), H, W, J);
    double val = a;
    const bool nyq = ((H & 1) == 0 && n1 == H / 2) || ((W & 1) == 0 && n2 == W / 2);
    if (nyq) {  // DFT partner (-n1 mod H, -n2 mod W)
      const int m1 = (H - n1) % H, m2 = (W - n2) % W;
      const double b = spectrum(d, freq(m1, H), freq(m2, W), H, W, J);
      val = sqrt(0.5 * (a * a + b * b));
    }
    bank[e] = static_cast<float>(val);
  }
}

// Column support of each filter on the half plane: the smallest and largest
// column index holding a non-zero value (the windows have compact support, so
// the spectra are exactly zero elsewhere).  One block per filter.
__global__ void k_filter_ranges(const float* __restrict__ bank, int H, int Wh, int2* __restrict__ ranges) {
  __shared__ int lo, hi;
  if (threadIdx.x == 0) {
    lo = Wh;
    hi = -1;
  }
  __syncthreads();
  const float* F = bank + static_cast<size_t>(blockIdx.x) * H * Wh;
  for (int c = threadIdx.x; c < Wh; c += blockDim.x) {
    bool nz = false;
    for (int r = 0; r < H && !nz; ++r) nz = F[static_cast<size_t>(r) * Wh + c] != 0.f;
    if (nz) {
      atomicMin(&lo, c);
      atomicMax(&hi, c);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) ranges[blockIdx.x] = make_int2(lo, hi);
}

__global__ void k_twiddles(float2* __restrict__ tw, int N) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < N; m += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(-2.0 * static_cast<double>(m) / static_cast<double>(N), &s, &c);
    tw[m] = make_float2(static_cast<float>(c), static_cast<float>(s));
  }
}

struct Codebook {
  float c[kMaxK * kMaxC];
};

// eq. computationOfs (p = 2) and its RGB form: s[k][r] = sum_ch (f[ch][r] - c[k][ch])^2.
__global__ void k_data_term(const float* __restrict__ f, int C, Codebook cb, int K, float* __restrict__ s, int P) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < P; r += gridDim.x * blockDim.x) {
    float fv[kMaxC];
#pragma unroll
    for (int ch = 0; ch < kMaxC; ++ch) fv[ch] = ch < C ? f[static_cast<size_t>(ch) * P + r] : 0.f;
    for (int k = 0; k < K; ++k) {
      float acc = 0.f;
#pragma unroll
      for (int ch = 0; ch < kMaxC; ++ch) {
        if (ch < C) {
          const float d = fv[ch] - cb.c[k * C + ch];
          acc = fmaf(d, d, acc);
        }
      }
      s[static_cast<size_t>(k) * P + r] = acc;
    }
  }
}

// Label = argmax_k w[k] (ties: lowest k), gap = largest - second largest.
__global__ void k_labels(const float* __restrict__ w, int K, int P, int* __restrict__ labels, float* __restrict__ gap) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < P; r += gridDim.x * blockDim.x) {
    int best = 0;
    float b1 = w[r], b2 = -INFINITY;
    for (int k = 1; k < K; ++k) {
      const float v = w[static_cast<size_t>(k) * P + r];
      if (v > b1) {
        b2 = b1;
        b1 = v;
        best = k;
      } else if (v > b2) {
        b2 = v;
      }
    }
    if (labels) labels[r] = best;
    if (gap) gap[r] = b1 - b2;
  }
}

__global__ void k_count_nonfinite(const float* __restrict__ x, long long n, int* __restrict__ count) {
  int c = 0;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x)
    c += isfinite(x[i]) ? 0 : 1;
  if (c) atomicAdd(count, c);
}

constexpr int kRedThreads = 256;

// Block-level FP64 sum in a fixed tree order.
__device__ double block_sum(double v) {
  __shared__ double buf[kRedThreads];
  buf[threadIdx.x] = v;
  __syncthreads();
  for (int s = kRedThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) buf[threadIdx.x] += buf[threadIdx.x + s];
    __syncthreads();
  }
  return buf[0];
}

template <int OP>  // 0: a*b, 1: (a-b)^2
__global__ void __launch_bounds__(kRedThreads) k_reduce2(const float* __restrict__ a, const float* __restrict__ b,
                                                         long long n, double* __restrict__ partial) {
  double acc = 0.0;
  for (long long i = blockIdx.x * static_cast<long long>(kRedThreads) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * kRedThreads) {
    const double x = a[i], y = b[i];
    acc += OP == 0 ? x * y : (x - y) * (x - y);
  }
  const double t = block_sum(acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

__global__ void __launch_bounds__(kRedThreads) k_sum_partials(const double* __restrict__ partial, int n,
                                                              double* __restrict__ out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += kRedThreads) acc += partial[i];
  const double t = block_sum(acc);
  if (threadIdx.x == 0) *out = t;
}

__global__ void k_sub(const float* __restrict__ a, const float* __restrict__ b, float* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x)
    out[i] = a[i] - b[i];
}

int grid_for(long long n, int threads, int cap = 4096) {
  long long g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return static_cast<int>(g);
}

int pow2_floor(int x) {
  int p = 1;
  while (p * 2 <= x) p *= 2;
  return p;
}

}  // namespace

bool make_geo(int H, int W, int J, Geo* g) {
  if (H < 8 || W < 8 || H > kMaxSide || W > kMaxSide || (W & 1)) return false;
  if (J < 1 || J > kMaxJ) return false;
  g->H = H;
  g->W = W;
  g->J = J;
  g->eta = (1 << (J + 2)) - 3;
  g->L = W / 2;
  g->Wh = W / 2 + 1;
  if (!make_plan(H, &g->planH) || !make_plan(g->L, &g->planL)) return false;
  int tc = pow2_floor(4096 / H);
  if (tc < 4) tc = 4;
  if (tc > 16) tc = 16;
  if (tc > g->Wh) tc = g->Wh;
  g->TC = tc;
  g->ntiles = (g->Wh + tc - 1) / tc;
  const int E = H * tc;
  const int per = (E + kColThreads - 1) / kColThreads;
  g->maxe = per <= 8 ? 8 : (per <= 16 ? 16 : 32);
  if (per > 32) return false;
  int rb = 4096 / g->L;
  if (rb < 1) rb = 1;
  if (rb > H) rb = H;
  g->RB = rb;
  g->twH = nullptr;
  g->twW = nullptr;
  g->bank = nullptr;
  g->ranges = nullptr;
  return true;
}

int filter_descs(int J, FilterDesc* out) {
  int n = 0;
  out[n++] = {0, 0, 0};
  for (int j = 0; j < J; ++j) {
    const int p = 1 << j;
    for (int k = -p + 1; k <= p - 1; ++k) out[n++] = {1, j, k};
    for (int k = -p + 1; k <= p - 1; ++k) out[n++] = {2, j, k};
    out[n++] = {3, j, -p};
    out[n++] = {3, j, p};
  }
  return n;
}

cudaError_t launch_twiddles(float2* tw, int N, cudaStream_t st) {
  k_twiddles<<<grid_for(N, 256), 256, 0, st>>>(tw, N);
  return cudaGetLastError();
}

cudaError_t launch_build_bank(float* bank, const Geo& g, const FilterDesc* descs_dev, cudaStream_t st) {
  const long long total = static_cast<long long>(g.eta) * g.H * g.Wh;
  k_build_bank<<<grid_for(total, 256, 152 * 16), 256, 0, st>>>(bank, descs_dev, g.H, g.W, g.Wh, g.J, g.eta);
  return cudaGetLastError();
}

cudaError_t launch_filter_ranges(const float* bank, const Geo& g, int2* ranges, cudaStream_t st) {
  k_filter_ranges<<<g.eta, 256, 0, st>>>(bank, g.H, g.Wh, ranges);
  return cudaGetLastError();
}

cudaError_t launch_data_term(const float* f, int C, const float* codebook_host, int K, float* s, int P,
                             cudaStream_t st) {
  Codebook cb{};
  for (int i = 0; i < K * C; ++i) cb.c[i] = codebook_host[i];
  k_data_term<<<grid_for(P, 256), 256, 0, st>>>(f, C, cb, K, s, P);
  return cudaGetLastError();
}

cudaError_t launch_labels(const float* w, int K, int P, int* labels, float* gap, cudaStream_t st) {
  k_labels<<<grid_for(P, 256), 256, 0, st>>>(w, K, P, labels, gap);
  return cudaGetLastError();
}

cudaError_t launch_count_nonfinite(const float* x, long n, int* count, cudaStream_t st) {
  k_count_nonfinite<<<grid_for(n, 256), 256, 0, st>>>(x, n, count);
  return cudaGetLastError();
}

cudaError_t launch_dot(const float* a, const float* b, long n, double* partial, int nblocks, double* out,
                       cudaStream_t st) {
  k_reduce2<0><<<nblocks, kRedThreads, 0, st>>>(a, b, n, partial);
  k_sum_partials<<<1, kRedThreads, 0, st>>>(partial, nblocks, out);
  return cudaGetLastError();
}

cudaError_t launch_sqdiff(const float* a, const float* b, long n, double* partial, int nblocks, double* out,
                          cudaStream_t st) {
  k_reduce2<1><<<nblocks, kRedThreads, 0, st>>>(a, b, n, partial);
  k_sum_partials<<<1, kRedThreads, 0, st>>>(partial, nblocks, out);
  return cudaGetLastError();
}

cudaError_t launch_sub(const float* a, const float* b, float* out, long n, cudaStream_t st) {
  k_sub<<<grid_for(n, 256), 256, 0, st>>>(a, b, out, n);
  return cudaGetLastError();
}

cudaError_t launch_sum_partials(const double* partial, int n, double* out, cudaStream_t st) {
  k_sum_partials<<<1, kRedThreads, 0, st>>>(partial, n, out);
  return cudaGetLastError();
}

}  // namespace shf

// Register-resident FFTs for power-of-two lengths N >= 8 (sm_103a fast path).
//
// A CTA transforms a batch of kB = 8 sequences of length N with N threads:
// thread (b = t % 8, tt = t / 8) holds v[k] = x_b[tt + k N/8], k = 0..7
// ("stride layout").  Each pass does radix-8 butterflies in registers (a
// radix-4 or radix-2 pass last when log2 N is not a multiple of 3); between
// passes the values go through shared memory at their Stockham positions,
// double-buffered so that one barrier per exchange suffices.  The result is
// again in the stride layout, in natural order.  Shared memory rows hold the
// 8 batch members of one index with a stride of kS = 9 float2, so both the
// batch-fast exchanges and index-fast staging from global memory are free of
// bank conflicts (up to one two-way conflict in some exchanges).
#pragma once

#include "shf_fft.cuh"

namespace shf {
namespace reg {

constexpr int kB = 8;
constexpr int kS = kB + 1;

__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n / 2); }

__host__ __device__ __forceinline__ int sidx(int i, int b) { return i * kS + b; }

// exp(S 2 pi i m / Ntab) from the table tw[m] = exp(-2 pi i m / Ntab).
template <int S>
__host__ __device__ __forceinline__ float2 twid(const float2* tw, int m) {
  float2 w = tw[m];
  if (S > 0) w.y = -w.y;
  return w;
}

// Butterflies of one pass of radix R with span Ns for thread tt (8/R
// butterflies per thread).  Input v in the stride layout; on return v[m +
// q (8/R)] holds output q of butterfly m.  tw has N*TWSTEP entries.
template <int N, int R, int S, int TWSTEP>
__host__ __device__ __forceinline__ void pass_bfly(float2 (&v)[8], int tt, int Ns, const float2* tw) {
  constexpr int M = 8 / R;
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const int j = tt + m * (N / 8);
    float2 x[R];
#pragma unroll
    for (int t = 0; t < R; ++t) x[t] = v[m + t * M];
    if (Ns > 1) {
      const int step = (j & (Ns - 1)) * (N / (Ns * R)) * TWSTEP;
#pragma unroll
      for (int t = 1; t < R; ++t) x[t] = c_mul(x[t], twid<S>(tw, t * step));
    }
    dft_small<R, S>(x);
#pragma unroll
    for (int q = 0; q < R; ++q) v[m + q * M] = x[q];
  }
}

// Writes the outputs of a (non-final) pass to their Stockham positions.
template <int N, int R>
__host__ __device__ __forceinline__ void pass_store(const float2 (&v)[8], int tt, int b, int Ns, float2* out) {
  constexpr int M = 8 / R;
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const int j = tt + m * (N / 8);
    const int o = (j / Ns) * Ns * R + (j & (Ns - 1));
#pragma unroll
    for (int q = 0; q < R; ++q) out[sidx(o + q * Ns, b)] = v[m + q * M];
  }
}

template <int N>
__host__ __device__ __forceinline__ void load_stride(float2 (&v)[8], int tt, int b, const float2* in) {
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = in[sidx(tt + k * (N / 8), b)];
}

template <int N>
struct Passes {
  static constexpr int LG = ilog2(N);
  static constexpr int P8 = LG / 3;
  static constexpr int REM = 1 << (LG % 3);
  static constexpr int NPASS = P8 + (REM > 1 ? 1 : 0);
  __host__ __device__ static constexpr int radix(int p) { return p < P8 ? 8 : REM; }
};

// Pass p of the transform (compile-time p): load (p > 0), butterflies, store
// (p < last).  Ns = product of the radices of passes 0..p-1.
template <int N, int S, int TWSTEP, int P>
__host__ __device__ __forceinline__ void run_pass(float2 (&v)[8], int tt, int b, const float2* in, float2* out,
                                                  const float2* tw) {
  constexpr int R = Passes<N>::radix(P);
  int Ns = 1;
#pragma unroll
  for (int p = 0; p < P; ++p) Ns *= Passes<N>::radix(p);
  if (P > 0) load_stride<N>(v, tt, b, in);
  pass_bfly<N, R, S, TWSTEP>(v, tt, Ns, tw);
  if (P < Passes<N>::NPASS - 1) pass_store<N, R>(v, tt, b, Ns, out);
}

#ifdef __CUDACC__
// The whole transform on the CTA's batch; buf0/buf1 hold N*kS float2 each.
// Starts with a barrier (the buffers may still be read by a previous
// transform) and ends with the result in v.
template <int N, int S, int TWSTEP>
__device__ __forceinline__ void fft(float2 (&v)[8], int tt, int b, float2* buf0, float2* buf1, const float2* tw) {
  constexpr int NP = Passes<N>::NPASS;
  if (NP > 1) __syncthreads();
  run_pass<N, S, TWSTEP, 0>(v, tt, b, nullptr, buf0, tw);
  if (NP > 1) {
    __syncthreads();
    run_pass<N, S, TWSTEP, (NP > 1 ? 1 : 0)>(v, tt, b, buf0, buf1, tw);
  }
  if (NP > 2) {
    __syncthreads();
    run_pass<N, S, TWSTEP, (NP > 2 ? 2 : 0)>(v, tt, b, buf1, buf0, tw);
  }
  if (NP > 3) {
    __syncthreads();
    run_pass<N, S, TWSTEP, (NP > 3 ? 3 : 0)>(v, tt, b, buf0, buf1, tw);
  }
}
#endif

}  // namespace reg
}  // namespace shf

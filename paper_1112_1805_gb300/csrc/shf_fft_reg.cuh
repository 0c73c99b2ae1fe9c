// Register-resident FFTs for lengths N = R 2^a with R in {1, 3, 5},
// 2^a >= 8 and N <= 2048 (sm_103a fast path).
//
// A CTA transforms a batch of KB (8, or 4 for N > 1024) sequences of length N
// with N KB / 8 threads: thread (b = t % KB, tt = t / KB) holds
// v[k] = x_b[tt + k N/8], k = 0..7 ("stride layout").  Stockham passes: for R > 1 a first pass of radix R,
// then radix-8 passes (a radix-4 or radix-2 pass last when log2(N/R) is not a
// multiple of 3).  A radix-8/4/2 pass does its butterflies in registers;
// between passes the values go through shared memory at their Stockham
// positions, double-buffered so that one barrier per exchange suffices.  The
// radix-R pass (span 1, so without twiddles) reads the natural-order input from
// shared memory and computes each of the thread's 8 outputs as an R-term sum:
// since N/8 is a multiple of R, all 8 outputs tt + k N/8 of a thread have the
// same DFT index q = tt mod R, so its R - 1 DFT weights are fixed per thread.
// The result is again in the stride layout, in natural order.  Shared memory
// rows hold the 8 batch members of one index (64 bytes); row i is stored at
// row i + (i >> 3) (one padding row after every 8), so that for powers of two
// the stride-layout reads, the Stockham writes of every pass and batch-fast
// staging all touch each bank the minimum number of times (checked by
// enumerating every access pattern), and every address is a per-thread base
// plus a compile-time offset.
#pragma once

#include "shf_fft.cuh"

namespace shf {
namespace reg {

constexpr int kB = 8;
constexpr int kS = kB;  // float2 per shared-memory row

__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n / 2); }
// Odd factor R of a supported length N = R 2^a.
__host__ __device__ constexpr int odd_part(int n) { return n % 3 == 0 ? 3 : (n % 5 == 0 ? 5 : 1); }
// Lengths of the register FFTs: R 2^a with R in {1, 3, 5}, 2^a >= 8, at most
// 1024 (rows and columns) or 2048 (columns, in batches of 4).
__host__ __device__ constexpr bool supported_upto(int n, int nmax) {
  return n >= 8 && n <= nmax && (n / odd_part(n)) % 8 == 0 && ((n / odd_part(n)) & (n / odd_part(n) - 1)) == 0;
}
__host__ __device__ constexpr bool supported(int n) { return supported_upto(n, 1024); }
__host__ __device__ constexpr bool supported_col(int n) { return supported_upto(n, 2048); }
// Columns per batch of the column transforms of height H.
__host__ __device__ constexpr int col_batch(int H) { return H > 1024 ? 4 : 8; }

// Padded row of index i in the batch layout, and the element offset.
__host__ __device__ constexpr int brow(int i) { return i + (i >> 3); }
template <int KB = kB>
__host__ __device__ __forceinline__ int sidx(int i, int b) {
  return brow(i) * KB + b;
}
// Rows a batch buffer of length N needs (index N included, for staging).
__host__ __device__ constexpr int batch_rows(int N) { return brow(N) + 1; }

// exp(S 2 pi i m / Ntab) from the table tw[m] = exp(-2 pi i m / Ntab).
template <int S>
__host__ __device__ __forceinline__ float2 twid(const float2* tw, int m) {
  float2 w = tw[m];
  if (S > 0) w.y = -w.y;
  return w;
}

template <int N>
struct Passes {
  static constexpr int R = odd_part(N);
  static constexpr int M = N / R;  // power-of-two part
  static constexpr int LG = ilog2(M);
  static constexpr int FIRST = R > 1 ? 1 : 0;  // passes of radix R (first)
  static constexpr int P8 = LG / 3;
  static constexpr int REM = 1 << (LG % 3);
  static constexpr int NPASS = FIRST + P8 + (REM > 1 ? 1 : 0);
  __host__ __device__ static constexpr int radix(int p) { return p < FIRST ? R : (p - FIRST < P8 ? 8 : REM); }
  __host__ __device__ static constexpr int span(int p) { return p == 0 ? 1 : span(p - 1) * radix(p - 1); }
  // offset of pass p's twiddles in the per-pass table: pass p (>= 1) holds
  // (radix - 1) * span entries, [t - 1][j mod span]
  __host__ __device__ static constexpr int twoff(int p) {
    return p <= 1 ? 0 : twoff(p - 1) + (radix(p - 1) - 1) * span(p - 1);
  }
  static constexpr int TWSIZE = twoff(NPASS) > 0 ? twoff(NPASS) : 1;
};

// cos and sin of 2 pi m / R for the radix-R first pass (R = 3 or 5).
template <int R>
__host__ __device__ __forceinline__ float2 unit_root(int m) {
  if (R == 3) {
    const float c = -0.5f, s = 0.86602540378443864676f;  // cos, sin of 2 pi / 3
    return m == 0 ? make_float2(1.f, 0.f) : (m == 1 ? make_float2(c, s) : make_float2(c, -s));
  }
  // cos, sin of 2 pi / 5 and 4 pi / 5
  const float c1 = 0.30901699437494742410f, s1 = 0.95105651629515357212f;
  const float c2 = -0.80901699437494742410f, s2 = 0.58778525229247312917f;
  switch (m) {
    case 0: return make_float2(1.f, 0.f);
    case 1: return make_float2(c1, s1);
    case 2: return make_float2(c2, s2);
    case 3: return make_float2(c2, -s2);
    default: return make_float2(c1, -s1);
  }
}

// The radix-R first pass (span 1): v[k] = y[tt + k N/8] with
// y[j R + q] = sum_t exp(S 2 pi i t q / R) x[j + t N/R]; the thread's
// q = tt mod R and j = tt / R + k N/(8R).  x is read from shared memory
// through idx(n).
template <int N, int S, typename Idx>
__host__ __device__ __forceinline__ void first_pass(float2 (&v)[8], int tt, const float2* x, Idx idx) {
  constexpr int R = Passes<N>::R;
  const int q = tt % R, j0 = tt / R;
  float2 c[R];
#pragma unroll
  for (int t = 0; t < R; ++t) {
    const float2 u = unit_root<R>((t * q) % R);
    c[t] = make_float2(u.x, static_cast<float>(S) * u.y);
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int j = j0 + k * (N / (8 * R));
    float2 a = x[idx(j)];
#pragma unroll
    for (int t = 1; t < R; ++t) {
      const float2 z = x[idx(j + t * (N / R))];
      a.x = fmaf(c[t].x, z.x, fmaf(-c[t].y, z.y, a.x));
      a.y = fmaf(c[t].x, z.y, fmaf(c[t].y, z.x, a.y));
    }
    v[k] = a;
  }
}

// Butterflies of one pass of radix R (8, 4 or 2) with span Ns for thread tt
// (8/R butterflies per thread).  Input v in the stride layout; on return
// v[m + q (8/R)] holds output q of butterfly m.  pt is this pass's part of
// the per-pass twiddle table.
template <int N, int R, int S, int Ns>
__host__ __device__ __forceinline__ void pass_bfly(float2 (&v)[8], int tt, const float2* pt) {
  constexpr int M = 8 / R;
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const int j = tt + m * (N / 8);
    float2 x[R];
#pragma unroll
    for (int t = 0; t < R; ++t) x[t] = v[m + t * M];
    if (Ns > 1) {
      const int k = j % Ns;
#pragma unroll
      for (int t = 1; t < R; ++t) x[t] = c_mul(x[t], twid<S>(pt, (t - 1) * Ns + k));
    }
    dft_small<R, S>(x);
#pragma unroll
    for (int q = 0; q < R; ++q) v[m + q * M] = x[q];
  }
}

// Writes the outputs of a (non-final) pass to their Stockham positions
// o + q Ns.  For Ns = 1 and for Ns a multiple of 8, brow(o + q Ns) =
// brow(o) + brow(q Ns): one base per butterfly plus constant offsets.
template <int N, int R, int Ns, int KB>
__host__ __device__ __forceinline__ void pass_store(const float2 (&v)[8], int tt, int b, float2* out) {
  constexpr int M = 8 / R;
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const int j = tt + m * (N / 8);
    const int o = (j / Ns) * Ns * R + (j % Ns);
    if (Ns == 1 || Ns % 8 == 0) {
      float2* p = out + brow(o) * KB + b;
#pragma unroll
      for (int q = 0; q < R; ++q) p[brow(q * Ns) * KB] = v[m + q * M];
    } else {
#pragma unroll
      for (int q = 0; q < R; ++q) out[sidx<KB>(o + q * Ns, b)] = v[m + q * M];
    }
  }
}

// Reads the stride layout; for N/8 a multiple of 8 the rows are brow(tt) +
// brow(k N/8).
template <int N, int KB>
__host__ __device__ __forceinline__ void load_stride(float2 (&v)[8], int tt, int b, const float2* in) {
  constexpr int T = N / 8;
  if (T % 8 == 0) {
    const float2* p = in + brow(tt) * KB + b;
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = p[brow(k * T) * KB];
  } else {
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = in[sidx<KB>(tt + k * T, b)];
  }
}

// Writes the stride layout to natural positions (the input of a radix-R
// first pass).
template <int N, int KB>
__host__ __device__ __forceinline__ void store_stride(const float2 (&v)[8], int tt, int b, float2* out) {
  constexpr int T = N / 8;
#pragma unroll
  for (int k = 0; k < 8; ++k) out[sidx<KB>(tt + k * T, b)] = v[k];
}

// Fills the per-pass twiddle table pt[TWSIZE] from the base table
// tw[m] = exp(-2 pi i m / (N TWSTEP)): entry (t - 1) Ns + k of pass p is
// exp(-2 pi i t k / (Ns R)), so that consecutive threads read consecutive
// entries.  `i0`/`stride` distribute the entries over the calling threads.
template <int N, int TWSTEP>
__host__ __device__ __forceinline__ void build_pass_twiddles(float2* pt, const float2* tw, int i0, int stride) {
  using PS = Passes<N>;
  for (int p = 1; p < PS::NPASS; ++p) {
    const int R = PS::radix(p), Ns = PS::span(p), off = PS::twoff(p);
    for (int e = i0; e < (R - 1) * Ns; e += stride) {
      const int t = 1 + e / Ns, k = e % Ns;
      pt[off + e] = tw[t * k * (N / (Ns * R)) * TWSTEP];
    }
  }
}

// Pass p >= FIRST (radix 8, 4 or 2) of the batch transform: load (when the
// previous pass stored), butterflies, store (p < last).
template <int N, int S, int P, int KB = kB>
__host__ __device__ __forceinline__ void run_pass(float2 (&v)[8], int tt, int b, const float2* in, float2* out,
                                                  const float2* pt) {
  using PS = Passes<N>;
  constexpr int R = PS::radix(P);
  constexpr int Ns = PS::span(P);
  if (P > PS::FIRST) load_stride<N, KB>(v, tt, b, in);
  pass_bfly<N, R, S, Ns>(v, tt, pt + PS::twoff(P));
  if (P < PS::NPASS - 1) pass_store<N, R, Ns, KB>(v, tt, b, out);
}

// ---------------------------------------------------------------------------
// Row-group variant: one sequence of length N is owned by T = N/8 consecutive
// threads (tt = its index in the group), with a private shared buffer in which
// element i lives at ridx(i) = i + (i >> 4).  That padding makes the
// stride-layout reads, the Stockham writes and contiguous staging touch each
// bank the minimum number of times for N = 32 .. 1024 (powers of two) except
// the second-pass writes at N = 128 (one extra wavefront), and keeps every
// address a per-thread base plus a compile-time offset.  Buffers need
// row_buf(N) entries (index N included, for the extra half-spectrum element).
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int ridx(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int row_buf(int N) { return ridx(N) + 1; }

struct RowIdx {
  __host__ __device__ int operator()(int i) const { return ridx(i); }
};

// Stockham writes: ridx(o + q Ns) = ridx(o) + ridx(q Ns) for Ns = 1, 8 and
// multiples of 16 (the spans of the stored radix-8 passes of powers of two).
template <int N, int R, int Ns>
__host__ __device__ __forceinline__ void rpass_store(const float2 (&v)[8], int tt, float2* out) {
  constexpr int M = 8 / R;
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const int j = tt + m * (N / 8);
    const int o = (j / Ns) * Ns * R + (j % Ns);
    if (R == 8 && (Ns == 1 || Ns == 8 || Ns % 16 == 0)) {
      float2* p = out + ridx(o);
#pragma unroll
      for (int q = 0; q < R; ++q) p[ridx(q * Ns)] = v[m + q * M];
    } else {
#pragma unroll
      for (int q = 0; q < R; ++q) out[ridx(o + q * Ns)] = v[m + q * M];
    }
  }
}

// Stride-layout reads: ridx(tt + k T) = base(tt) + ridx(k T) with base = ridx(tt)
// for T a multiple of 16, and general addressing otherwise.
template <int N>
__host__ __device__ __forceinline__ void rload_stride(float2 (&v)[8], int tt, const float2* in) {
  constexpr int T = N / 8;
  if (T % 16 == 0) {
    const float2* p = in + ridx(tt);
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = p[ridx(k * T)];
  } else if (T < 16 && (T & (T - 1)) == 0) {  // T = 1, 2, 4, 8: tt + k T < 16 (k T) + tt, no carry into i >> 4
    const float2* p = in + tt;
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = p[ridx(k * T)];
  } else {
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = in[ridx(tt + k * T)];
  }
}

template <int N>
__host__ __device__ __forceinline__ void rstore_stride(const float2 (&v)[8], int tt, float2* out) {
  constexpr int T = N / 8;
#pragma unroll
  for (int k = 0; k < 8; ++k) out[ridx(tt + k * T)] = v[k];
}

template <int N, int S, int P>
__host__ __device__ __forceinline__ void rrun_pass(float2 (&v)[8], int tt, const float2* in, float2* out,
                                                   const float2* pt) {
  using PS = Passes<N>;
  constexpr int R = PS::radix(P);
  constexpr int Ns = PS::span(P);
  if (P > PS::FIRST) rload_stride<N>(v, tt, in);
  pass_bfly<N, R, S, Ns>(v, tt, pt + PS::twoff(P));
  if (P < PS::NPASS - 1) rpass_store<N, R, Ns>(v, tt, out);
}

// Whether row groups of T threads tile warps exactly (T divides 32, or is a
// multiple of 32).  Groups of other sizes (3 2^a or 5 2^a threads, a < 5)
// are packed back to back over the CTA's threads.
__host__ __device__ constexpr bool tiles_warps(int T) { return 32 % T == 0 || T % 32 == 0; }

#ifdef __CUDACC__
// Barrier of a row group: the warp when the group fits in it (every lane of
// the warp takes part), the named barrier `id` over the group's warps when
// it is whole warps, and the CTA's barrier when groups are packed across
// warps (every group of the CTA then takes part).
template <int T>
__device__ __forceinline__ void group_sync(int id) {
  if (!tiles_warps(T)) {
    __syncthreads();
  } else if (T <= 32) {
    __syncwarp();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(T) : "memory");
  }
}

// The whole transform of one sequence by its row group; result in v.  Starts
// with a barrier (the buffers may still be read by a previous transform).
template <int N, int S>
__device__ __forceinline__ void row_fft(float2 (&v)[8], int tt, float2* buf0, float2* buf1, const float2* pt,
                                        int bar_id) {
  using PS = Passes<N>;
  constexpr int NP = PS::NPASS;
  constexpr int T = N / 8;
  if (PS::FIRST) {
    group_sync<T>(bar_id);
    rstore_stride<N>(v, tt, buf1);
    group_sync<T>(bar_id);
    first_pass<N, S>(v, tt, buf1, RowIdx());
    rrun_pass<N, S, (NP > 1 ? 1 : 0)>(v, tt, nullptr, buf0, pt);  // v already in the stride layout
    if (NP > 2) {
      group_sync<T>(bar_id);
      rrun_pass<N, S, (NP > 2 ? 2 : 0)>(v, tt, buf0, buf1, pt);
    }
    if (NP > 3) {
      group_sync<T>(bar_id);
      rrun_pass<N, S, (NP > 3 ? 3 : 0)>(v, tt, buf1, buf0, pt);
    }
    if (NP > 4) {
      group_sync<T>(bar_id);
      rrun_pass<N, S, (NP > 4 ? 4 : 0)>(v, tt, buf0, buf1, pt);
    }
    return;
  }
  if (NP > 1) group_sync<T>(bar_id);
  rrun_pass<N, S, 0>(v, tt, nullptr, buf0, pt);
  if (NP > 1) {
    group_sync<T>(bar_id);
    rrun_pass<N, S, (NP > 1 ? 1 : 0)>(v, tt, buf0, buf1, pt);
  }
  if (NP > 2) {
    group_sync<T>(bar_id);
    rrun_pass<N, S, (NP > 2 ? 2 : 0)>(v, tt, buf1, buf0, pt);
  }
  if (NP > 3) {
    group_sync<T>(bar_id);
    rrun_pass<N, S, (NP > 3 ? 3 : 0)>(v, tt, buf0, buf1, pt);
  }
}

// The same with one buffer: every exchange reads the stored values and waits
// for the whole group before the next stores.  Starts with a barrier.
template <int N, int S, int P>
__device__ __forceinline__ void rpass1(float2 (&v)[8], int tt, float2* buf, const float2* pt, int bar_id) {
  using PS = Passes<N>;
  constexpr int R = PS::radix(P);
  constexpr int Ns = PS::span(P);
  constexpr int T = N / 8;
  if (P > PS::FIRST) {
    group_sync<T>(bar_id);
    rload_stride<N>(v, tt, buf);
  }
  pass_bfly<N, R, S, Ns>(v, tt, pt + PS::twoff(P));
  if (P < PS::NPASS - 1) {
    group_sync<T>(bar_id);
    rpass_store<N, R, Ns>(v, tt, buf);
  }
}

template <int N, int S>
__device__ __forceinline__ void row_fft1(float2 (&v)[8], int tt, float2* buf, const float2* pt, int bar_id) {
  using PS = Passes<N>;
  constexpr int NP = PS::NPASS;
  constexpr int T = N / 8;
  if (PS::FIRST) {
    group_sync<T>(bar_id);
    rstore_stride<N>(v, tt, buf);
    group_sync<T>(bar_id);
    first_pass<N, S>(v, tt, buf, RowIdx());
  }
  if (PS::FIRST < NP) rpass1<N, S, (PS::FIRST < NP ? PS::FIRST : 0)>(v, tt, buf, pt, bar_id);
  if (PS::FIRST + 1 < NP) rpass1<N, S, (PS::FIRST + 1 < NP ? PS::FIRST + 1 : 0)>(v, tt, buf, pt, bar_id);
  if (PS::FIRST + 2 < NP) rpass1<N, S, (PS::FIRST + 2 < NP ? PS::FIRST + 2 : 0)>(v, tt, buf, pt, bar_id);
  if (PS::FIRST + 3 < NP) rpass1<N, S, (PS::FIRST + 3 < NP ? PS::FIRST + 3 : 0)>(v, tt, buf, pt, bar_id);
}
#endif

#ifdef __CUDACC__
template <int KB>
struct BatchIdx {
  int b;
  __device__ int operator()(int i) const { return sidx<KB>(i, b); }
};

// The whole transform on the CTA's batch; buf0/buf1 hold batch_rows(N)*KB
// float2 each.  Starts with a barrier (the buffers may still be read by a
// previous transform) and ends with the result in v.
template <int N, int S, int KB = kB>
__device__ __forceinline__ void fft(float2 (&v)[8], int tt, int b, float2* buf0, float2* buf1, const float2* pt) {
  using PS = Passes<N>;
  constexpr int NP = PS::NPASS;
  if (PS::FIRST) {
    __syncthreads();
    store_stride<N, KB>(v, tt, b, buf1);
    __syncthreads();
    first_pass<N, S>(v, tt, buf1, BatchIdx<KB>{b});
    run_pass<N, S, (NP > 1 ? 1 : 0), KB>(v, tt, b, nullptr, buf0, pt);  // v already in the stride layout
    if (NP > 2) {
      __syncthreads();
      run_pass<N, S, (NP > 2 ? 2 : 0), KB>(v, tt, b, buf0, buf1, pt);
    }
    if (NP > 3) {
      __syncthreads();
      run_pass<N, S, (NP > 3 ? 3 : 0), KB>(v, tt, b, buf1, buf0, pt);
    }
    if (NP > 4) {
      __syncthreads();
      run_pass<N, S, (NP > 4 ? 4 : 0), KB>(v, tt, b, buf0, buf1, pt);
    }
    return;
  }
  if (NP > 1) __syncthreads();
  run_pass<N, S, 0, KB>(v, tt, b, nullptr, buf0, pt);
  if (NP > 1) {
    __syncthreads();
    run_pass<N, S, (NP > 1 ? 1 : 0), KB>(v, tt, b, buf0, buf1, pt);
  }
  if (NP > 2) {
    __syncthreads();
    run_pass<N, S, (NP > 2 ? 2 : 0), KB>(v, tt, b, buf1, buf0, pt);
  }
  if (NP > 3) {
    __syncthreads();
    run_pass<N, S, (NP > 3 ? 3 : 0), KB>(v, tt, b, buf0, buf1, pt);
  }
}
#endif

}  // namespace reg
}  // namespace shf

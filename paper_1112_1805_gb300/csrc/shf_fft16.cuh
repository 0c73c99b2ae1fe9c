// Register FFTs with 16 values per thread for the rows of the v-step, lengths
// N = 2^a with 64 <= N <= 1024 (sm_103a fast path).
//
// A row group of T = N/16 threads (4, 8, 16 or 32: whole fractions of a warp;
// 64 for N = 1024: two warps) transforms one sequence; thread tt holds v[k] = x[tt + k T], k = 0..15
// ("stride layout").  Stockham passes of radix 16 (spans 1, 16, ...) and, when
// log2 N is not a multiple of 4, a last pass of radix 2, 4 or 8 in which each
// thread does 16/R butterflies.  N = 256 = 16 * 16 thus needs one exchange
// through shared memory, where the radix-8 transform of 8 values per thread
// needs two.  A radix-16 butterfly is a 4 x 4 decomposition in registers
// (twiddles of the 16th roots of unity are constants).
//
// The exchange buffer of a group stores element i at ridx(i) = i + (i >> 4).
// With 64-bit shared accesses served per half-warp, every access pattern used
// here touches 16 distinct bank pairs within a half-warp: the span-1 stores
// write i = 16 tt + q at 17 tt + q, the stride reads i = tt + k T are
// consecutive in tt, and the span-16 stores of N = 512 write blocks of 16
// consecutive indices.  Groups of T < 16 threads share a half-warp; their
// buffers are placed T float2 apart modulo 16 by the caller.
#pragma once

#include "shf_fft_reg.cuh"

namespace shf {
namespace r16 {

using reg::ilog2;
using reg::ridx;

template <int N>
struct Passes {
  static_assert(N >= 32 && N <= 2048 && (N & (N - 1)) == 0, "radix-16 FFT: N = 2^a, 32 <= N <= 2048");
  static constexpr int T = N / 16;                        // threads of a group
  static constexpr int LG = ilog2(N);
  static constexpr int N16 = LG / 4;                      // radix-16 passes (first)
  static constexpr int REM = 1 << (LG % 4);               // radix of the last pass (1: none)
  static constexpr int NPASS = N16 + (REM > 1 ? 1 : 0);
  __host__ __device__ static constexpr int radix(int p) { return p < N16 ? 16 : REM; }
  __host__ __device__ static constexpr int span(int p) { return p == 0 ? 1 : span(p - 1) * radix(p - 1); }
  // offset of pass p's twiddles (p >= 1): (radix - 1) * span entries, [t - 1][k]
  __host__ __device__ static constexpr int twoff(int p) {
    return p <= 1 ? 0 : twoff(p - 1) + (radix(p - 1) - 1) * span(p - 1);
  }
  static constexpr int TWSIZE = twoff(NPASS) > 0 ? twoff(NPASS) : 1;
};

// a * (c + i s)
__host__ __device__ __forceinline__ float2 cmul_cs(float2 a, float c, float s) {
  return make_float2(a.x * c - a.y * s, a.x * s + a.y * c);
}

// In-place 16-point DFT V_q = sum_t v_t exp(S 2 pi i t q / 16), natural order
// in and out: DFT-4 over a of v[4a + b] for each b, twiddles
// exp(S 2 pi i b q1 / 16), DFT-4 over b for each q1, then the 4 x 4 transpose
// (a renaming of registers).
template <int S>
__host__ __device__ __forceinline__ void dft16(float2 (&v)[16]) {
  constexpr float C1 = 0.92387953251128675613f;  // cos(pi/8)
  constexpr float S1 = 0.38268343236508977173f;  // sin(pi/8)
  constexpr float RH = 0.70710678118654752440f;  // cos(pi/4)
  const float s = static_cast<float>(S);
#pragma unroll
  for (int b = 0; b < 4; ++b) dft4_vals<S>(v[b], v[4 + b], v[8 + b], v[12 + b]);
  // slot 4 q1 + b holds y_b(q1); multiply by w^(b q1), w = exp(S 2 pi i / 16)
  v[5] = cmul_cs(v[5], C1, s * S1);     // w^1
  v[6] = cmul_cs(v[6], RH, s * RH);     // w^2
  v[7] = cmul_cs(v[7], S1, s * C1);     // w^3
  v[9] = cmul_cs(v[9], RH, s * RH);     // w^2
  v[10] = c_mul_si<S>(v[10]);           // w^4 = S i
  v[11] = cmul_cs(v[11], -RH, s * RH);  // w^6
  v[13] = cmul_cs(v[13], S1, s * C1);   // w^3
  v[14] = cmul_cs(v[14], -RH, s * RH);  // w^6
  v[15] = cmul_cs(v[15], -C1, -s * S1); // w^9
#pragma unroll
  for (int q1 = 0; q1 < 4; ++q1) dft4_vals<S>(v[4 * q1], v[4 * q1 + 1], v[4 * q1 + 2], v[4 * q1 + 3]);
  // slot 4 q1 + q2 holds V(q1 + 4 q2)
  float2 t;
  t = v[1], v[1] = v[4], v[4] = t;
  t = v[2], v[2] = v[8], v[8] = t;
  t = v[3], v[3] = v[12], v[12] = t;
  t = v[6], v[6] = v[9], v[9] = t;
  t = v[7], v[7] = v[13], v[13] = t;
  t = v[11], v[11] = v[14], v[14] = t;
}

template <int R, int S>
__host__ __device__ __forceinline__ void dft_r(float2* x) {
  if constexpr (R == 16) {
    dft16<S>(*reinterpret_cast<float2(*)[16]>(x));
  } else {
    dft_small<R, S>(x);
  }
}

// Butterflies of pass P for thread tt: 16/R butterflies of radix R; butterfly
// m (index j = tt + m T) takes v[m + t (16/R)], t = 0..R-1, multiplies by the
// twiddles exp(S 2 pi i t (j mod Ns) / (Ns R)) from the per-pass table pt and
// leaves output q in v[m + q (16/R)].
template <int N, int P, int S>
__host__ __device__ __forceinline__ void pass_bfly(float2 (&v)[16], int tt, const float2* pt) {
  using PS = Passes<N>;
  constexpr int R = PS::radix(P), Ns = PS::span(P), M = 16 / R, T = PS::T;
#pragma unroll
  for (int m = 0; m < M; ++m) {
    float2 x[R];
#pragma unroll
    for (int t = 0; t < R; ++t) x[t] = v[m + t * M];
    if constexpr (Ns > 1) {
      const int k = (tt + m * T) & (Ns - 1);
      const float2* p = pt + PS::twoff(P) + k;
#pragma unroll
      for (int t = 1; t < R; ++t) x[t] = c_mul(x[t], reg::twid<S>(p, (t - 1) * Ns));
    }
    dft_r<R, S>(x);
#pragma unroll
    for (int q = 0; q < R; ++q) v[m + q * M] = x[q];
  }
}

// Stockham writes of a radix-16 pass: output q of butterfly j goes to
// o + q Ns with o = (j / Ns) Ns 16 + (j mod Ns); since o mod 16 + (q Ns) mod 16
// < 16, ridx(o + q Ns) = ridx(o) + ridx(q Ns).
template <int N, int P>
__host__ __device__ __forceinline__ void pass_store(const float2 (&v)[16], int tt, float2* out) {
  using PS = Passes<N>;
  constexpr int R = PS::radix(P), Ns = PS::span(P);
  static_assert(R == 16, "only radix-16 passes are followed by an exchange");
  const int o = (tt / Ns) * Ns * 16 + (tt & (Ns - 1));
  float2* p = out + ridx(o);
#pragma unroll
  for (int q = 0; q < 16; ++q) p[ridx(q * Ns)] = v[q];
}

// Stride-layout reads v[k] = x[tt + k T]: ridx(tt + k T) = ridx(tt) + ridx(k T)
// for T a multiple of 16, and tt + ridx(k T) for T dividing 16 (tt < T).
template <int N>
__host__ __device__ __forceinline__ void load_stride(float2 (&v)[16], int tt, const float2* in) {
  constexpr int T = Passes<N>::T;
  const float2* p = in + (T % 16 == 0 ? ridx(tt) : tt);
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = p[ridx(k * T)];
}

// Per-pass twiddle table pt[TWSIZE] from the base table
// tw[m] = exp(-2 pi i m / (N TWSTEP)): entry twoff(p) + (t - 1) Ns + k of pass
// p is exp(-2 pi i t k / (Ns R)).
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

// Batch variants for the column transforms: a CTA transforms KB columns of
// length N; thread (b, tt) holds v[k] = x_b[tt + k T] (T = N/16), and element i
// of column b lives at (ridx(i)) KB + b of the exchange buffer.  Within a
// half-warp (KB = 8: two consecutive tt; KB = 4: four) the stride reads are
// consecutive rows and the span-1 stores are rows 17 apart, i.e. 8 (or 4)
// banks apart per row: no bank conflicts.
template <int N, int P, int KB>
__host__ __device__ __forceinline__ void bpass_store(const float2 (&v)[16], int tt, int b, float2* out) {
  using PS = Passes<N>;
  constexpr int R = PS::radix(P), Ns = PS::span(P);
  static_assert(R == 16, "only radix-16 passes are followed by an exchange");
  const int o = (tt / Ns) * Ns * 16 + (tt & (Ns - 1));
  float2* p = out + ridx(o) * KB + b;
#pragma unroll
  for (int q = 0; q < 16; ++q) p[ridx(q * Ns) * KB] = v[q];
}

template <int N, int KB>
__host__ __device__ __forceinline__ void bload_stride(float2 (&v)[16], int tt, int b, const float2* in) {
  constexpr int T = Passes<N>::T;
  const float2* p = in + (T % 16 == 0 ? ridx(tt) : tt) * KB + b;
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = p[ridx(k * T) * KB];
}

// Rows of an exchange buffer of a length-N batch transform.
__host__ __device__ constexpr int brows16(int N) { return ridx(N) + 1; }

// Real rows of length W = 2L as complex rows of length L (z[n] = x[2n] + i x[2n+1]).
// In the stride layout index L - (tt + k T) is register 15 - k of lane
// (T - tt) mod T, and for lane 0 its own register 16 - k (k >= 1; index L for
// k = 0): the pairings of the packing are warp shuffles.

// Step k (0..7) of the in-place inverse packing
// Z[n] = (X_n + conj X_{L-n}) + i e^{+2 pi i n/W} (X_n - conj X_{L-n}): registers
// k and 15 - k (holding X at n = tt + k T and tt + (15 - k) T) become Z.  ra, rb
// are the partner lane's registers 15 - k and k as they were before this step
// (unused on lane 0).  Lane 0 pairs registers k and 16 - k instead; its register
// 16 - k was overwritten at step k - 1, so it is carried in `prev` (X_L before
// step 0).  tw[m] = exp(-2 pi i m / W).
template <int L>
__host__ __device__ __forceinline__ void pack_step(float2 (&v)[16], int k, int tt, float2 ra, float2 rb, float2& prev,
                                                   const float2* tw) {
  constexpr int T = L / 16;
  const int k2 = 15 - k;
  if (tt == 0) {
    ra = prev;      // X_{L - T k}
    rb = v[k + 1];  // X_{L - T k2}, not yet overwritten
  }
  prev = v[k2];
  const float2 a1 = v[k], a2 = v[k2];
  {
    const float2 c = c_conj(ra);
    const float2 s2 = c_add(a1, c), d = c_sub(a1, c);
    v[k] = pack_combine(s2, d, tw[tt + k * T]);
  }
  {
    const float2 c = c_conj(rb);
    const float2 s2 = c_add(a2, c), d = c_sub(a2, c);
    v[k2] = pack_combine(s2, d, tw[tt + k2 * T]);
  }
}

// Forward unpacking X[i] = 1/2 [(Z_i + conj Z_{L-i}) - i e^{-2 pi i i/W} (Z_i - conj Z_{L-i})]
// at i = tt + q T from register q (Z_i) and r, the partner lane's register
// 15 - q (on lane 0 Z_{L-i} is its own register (16 - q) mod 16).  X[L] is
// Re Z_0 - Im Z_0 (e^{-i pi} = -1), formed by lane 0.
template <int L>
__host__ __device__ __forceinline__ float2 unpack_value(const float2 (&v)[16], int q, int tt, float2 r,
                                                        const float2* tw) {
  constexpr int T = L / 16;
  const float2 zb = tt == 0 ? v[(16 - q) & 15] : r;
  const float2 c = c_conj(zb);
  const float2 s2 = c_add(v[q], c), d = c_sub(v[q], c);
  return unpack_combine(s2, d, tw[tt + q * T]);
}

// Two real rows a, b of length W as one complex row z = a + i b, transformed
// with length W.  Spectrum of z from the half spectra Xa, Xb (k = 0 .. W/2):
// Z[n] = Xa[n] + i Xb[n] for n <= W/2 and Z[n] = conj Xa[W-n] + i conj Xb[W-n]
// above; `upper` selects the second form (xa, xb then hold Xa[W-n], Xb[W-n]).
__host__ __device__ __forceinline__ float2 pair_pack(float2 xa, float2 xb, bool upper) {
  return upper ? make_float2(xa.x + xb.y, xb.x - xa.y) : make_float2(xa.x - xb.y, xa.y + xb.x);
}

// Half spectra of the rows from D = FFT(d_a + i d_b): Xa[k] = (D_k + conj D_{W-k})/2,
// Xb[k] = (D_k - conj D_{W-k})/(2i); dm = D_{W-k}.
__host__ __device__ __forceinline__ void pair_unpack(float2 dk, float2 dm, float2& xa, float2& xb) {
  const float2 c = c_conj(dm);
  const float2 s2 = c_add(dk, c), t = c_sub(dk, c);
  xa = c_mul2(s2, make_float2(0.5f, 0.5f));
  xb = make_float2(0.5f * t.y, -0.5f * t.x);
}

// The register of the partner lane holding D_{W-k} for k = tt + q T (stride
// layout of a length-N = 16 T transform): register 15 - q of lane (T - tt)
// mod T, or, on lane 0, its own register (16 - q) mod 16 (given as `own`).
__host__ __device__ __forceinline__ float2 pair_partner(int tt, float2 from_partner, float2 own) {
  return tt == 0 ? own : from_partner;
}

#ifdef __CUDACC__
// Barrier of a row group: the warp for T <= 32 (all lanes of the warp take
// part), else the named barrier `id` over the group's T threads (whole warps).
template <int N>
__device__ __forceinline__ void group_sync(int id) {
  if constexpr (Passes<N>::T <= 32) {
    __syncwarp();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(Passes<N>::T) : "memory");
  }
}

// The transform of a CTA's KB columns (every thread of the CTA takes part;
// two buffers, one CTA barrier per exchange plus one before the first, which
// also covers the previous transform's reads); result in v, in the stride
// layout.
template <int N, int S, int KB>
__device__ __forceinline__ void batch_fft(float2 (&v)[16], int tt, int b, float2* buf0, float2* buf1,
                                          const float2* pt) {
  using PS = Passes<N>;
  pass_bfly<N, 0, S>(v, tt, pt);
  if constexpr (PS::NPASS > 1) {
    __syncthreads();
    bpass_store<N, 0, KB>(v, tt, b, buf0);
    __syncthreads();
    bload_stride<N, KB>(v, tt, b, buf0);
    pass_bfly<N, (PS::NPASS > 1 ? 1 : 0), S>(v, tt, pt);
  }
  if constexpr (PS::NPASS > 2) {
    bpass_store<N, (PS::NPASS > 2 ? 1 : 0), KB>(v, tt, b, buf1);
    __syncthreads();
    bload_stride<N, KB>(v, tt, b, buf1);
    pass_bfly<N, (PS::NPASS > 2 ? 2 : 0), S>(v, tt, pt);
  }
}

// The transform of one sequence by its row group; result in v, in the stride
// layout.  The first exchange starts with a barrier: the buffer may still be
// read by a previous transform.
template <int N, int S>
__device__ __forceinline__ void row_fft(float2 (&v)[16], int tt, float2* buf, const float2* pt, int bar_id) {
  using PS = Passes<N>;
  pass_bfly<N, 0, S>(v, tt, pt);
  if constexpr (PS::NPASS > 1) {
    group_sync<N>(bar_id);
    pass_store<N, 0>(v, tt, buf);
    group_sync<N>(bar_id);
    load_stride<N>(v, tt, buf);
    pass_bfly<N, (PS::NPASS > 1 ? 1 : 0), S>(v, tt, pt);
  }
  if constexpr (PS::NPASS > 2) {
    group_sync<N>(bar_id);
    pass_store<N, (PS::NPASS > 2 ? 1 : 0)>(v, tt, buf);
    group_sync<N>(bar_id);
    load_stride<N>(v, tt, buf);
    pass_bfly<N, (PS::NPASS > 2 ? 2 : 0), S>(v, tt, pt);
  }
}
#endif

}  // namespace r16
}  // namespace shf

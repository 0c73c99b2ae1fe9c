// Register FFTs with V values per thread: for the lengths with an odd factor,
// L = 3 2^a (V = 12) and L = 5 2^a (V = 20), and for the row length
// 1024 = 32 x 32 (V = 32), split as L = V T over T threads (a power of two):
// the v-step's rows with T = 2 .. 32 (a group never leaves its warp and every
// barrier is __syncwarp), and the fan's and gather's columns (V = 12, 20) in
// batches of KB columns with T = 2 .. 128 (CTA barriers).
//
// Thread tt holds v[k] = x[tt + k T], k = 0..V-1 ("stride layout", as in
// shf_fft16.cuh).  Stockham passes: first one of radix V (span 1: no
// twiddles; a V = R x 4 decomposition in registers with R = 3, 5 or 8 and the
// V-th roots of unity as constants), then radix-4 passes and, when log2 T is
// odd, a last radix-2 pass, in which each thread does V/4 (or V/2)
// butterflies; for V = 32 one more radix-32 pass, one butterfly per thread.
// The exchange buffers are laid out per pass so that a half-warp's 64-bit
// accesses spread over the 16 bank pairs (xidx, bxidx).  The real-row packing
// pairs index n = tt + k T with L - n, which is register V - 1 - k of lane
// (T - tt) mod T (lane 0: its own register V - k, or X_L for k = 0): the
// pairings are warp shuffles.
#pragma once

#include "shf_fft16.cuh"

namespace shf {
namespace rv {

using reg::ilog2;
using reg::ridx;

// Values per thread for a half width L (0: no V-value transform); 32 for the
// power of two 1024 = 32 x 32, split as two radix-32 passes over one warp.
__host__ __device__ constexpr int vals_for(int L) {
  return reg::odd_part(L) == 3 ? 12 : (reg::odd_part(L) == 5 ? 20 : (L == 1024 ? 32 : 0));
}
__host__ __device__ constexpr bool pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }
// Lengths with a V-value transform of T = L / V threads per sequence, a power
// of two in [2, tmax]: rows up to 32 (one warp), columns up to 128 (the CTA's
// barriers).
__host__ __device__ constexpr bool supported_upto(int L, int tmax) {
  return vals_for(L) > 0 && L % vals_for(L) == 0 && pow2(L / vals_for(L)) && L / vals_for(L) >= 2 &&
         L / vals_for(L) <= tmax;
}
__host__ __device__ constexpr bool supported(int L) { return supported_upto(L, 32); }
__host__ __device__ constexpr bool supported_col(int H) { return supported_upto(H, 128) && vals_for(H) != 32; }

template <int L>
struct Passes {
  static_assert(supported_upto(L, 128), "V-value FFT: L = 12 T or 20 T, T = 2^a in [2, 128], or L = 32 x 32");
  static constexpr int V = vals_for(L);
  static constexpr int T = L / V;
  static constexpr bool SQ = V == 32;             // 32 x 32: a second radix-32 pass, one butterfly per thread
  static constexpr int LGT = ilog2(T);
  static constexpr int N4 = SQ ? 0 : LGT / 2;     // radix-4 passes after the first
  static constexpr int REM = (!SQ && LGT % 2) ? 2 : 1;  // a last radix-2 pass
  static constexpr int NPASS = SQ ? 2 : 1 + N4 + (REM > 1 ? 1 : 0);
  __host__ __device__ static constexpr int radix(int p) {
    return p == 0 ? V : (SQ ? T : (p - 1 < N4 ? 4 : REM));
  }
  __host__ __device__ static constexpr int span(int p) { return p == 0 ? 1 : span(p - 1) * radix(p - 1); }
  // offset of pass p's twiddles (p >= 1): (radix - 1) * span entries, [t - 1][k]
  __host__ __device__ static constexpr int twoff(int p) {
    return p <= 1 ? 0 : twoff(p - 1) + (radix(p - 1) - 1) * span(p - 1);
  }
  static constexpr int TWSIZE = twoff(NPASS) > 0 ? twoff(NPASS) : 1;
};

// cos and sin of 2 pi m / V for the internal twiddles of a radix-V pass
// (m < V: 12, 20 or 32), from the values of sin and cos at multiples of 30,
// 18 and 11.25 degrees.
template <int V>
__host__ __device__ __forceinline__ float2 root(int m) {
  if (V == 32) {
    const float2 q[8] = {make_float2(1.f, 0.f),
                         make_float2(0.98078528040323044913f, 0.19509032201612826785f),
                         make_float2(0.92387953251128675613f, 0.38268343236508977173f),
                         make_float2(0.83146961230254523708f, 0.55557023301960222474f),
                         make_float2(0.70710678118654752440f, 0.70710678118654752440f),
                         make_float2(0.55557023301960222474f, 0.83146961230254523708f),
                         make_float2(0.38268343236508977173f, 0.92387953251128675613f),
                         make_float2(0.19509032201612826785f, 0.98078528040323044913f)};  // 11.25 r degrees
    const int r = m % 8, s = m / 8;  // m * 11.25 = 90 s + 11.25 r
    float2 a = q[r];
    for (int i = 0; i < s; ++i) a = make_float2(-a.y, a.x);
    return a;
  }
  constexpr float H3 = 0.86602540378443864676f;  // cos 30, sin 60
  constexpr float C18 = 0.95105651629515357212f, S18 = 0.30901699437494742410f;
  constexpr float C36 = 0.80901699437494742410f, S36 = 0.58778525229247312917f;
  if (V == 12) {
    const float2 q[3] = {make_float2(1.f, 0.f), make_float2(H3, 0.5f), make_float2(0.5f, H3)};  // 0, 30, 60 degrees
    const int r = m % 3, s = m / 3;  // m * 30 = 90 s + 30 r
    float2 a = q[r];
    for (int i = 0; i < s; ++i) a = make_float2(-a.y, a.x);  // + 90 degrees
    return a;
  }
  const float2 q[5] = {make_float2(1.f, 0.f), make_float2(C18, S18), make_float2(C36, S36), make_float2(S36, C36),
                       make_float2(S18, C18)};  // 0, 18, 36, 54, 72 degrees
  const int r = m % 5, s = m / 5;               // m * 18 = 90 s + 18 r
  float2 a = q[r];
  for (int i = 0; i < s; ++i) a = make_float2(-a.y, a.x);
  return a;
}

// In-place V-point DFT V_q = sum_t v_t exp(S 2 pi i t q / V), natural order in
// and out, V = R x 4: DFT-R over t1 of v[4 t1 + t2] for each t2, twiddles
// exp(S 2 pi i t2 q1 / V), DFT-4 over t2 for each q1; V_{q1 + R q2} lands in
// register q1 + R q2.
template <int V, int S>
__host__ __device__ __forceinline__ void dftv(float2 (&v)[V]) {
  constexpr int R = V / 4;
  float2 y[V];  // y[t2 R + q1]
#pragma unroll
  for (int t2 = 0; t2 < 4; ++t2) {
    float2 x[R];
#pragma unroll
    for (int t1 = 0; t1 < R; ++t1) x[t1] = v[4 * t1 + t2];
    dft_small<R, S>(x);
#pragma unroll
    for (int q1 = 0; q1 < R; ++q1) {
      if (t2 * q1 == 0) {
        y[t2 * R + q1] = x[q1];
      } else {
        float2 w = root<V>(t2 * q1);
        if (S < 0) w.y = -w.y;
        y[t2 * R + q1] = c_mul(x[q1], w);
      }
    }
  }
#pragma unroll
  for (int q1 = 0; q1 < R; ++q1) {
    float2 a = y[q1], b = y[R + q1], c = y[2 * R + q1], d = y[3 * R + q1];
    dft4_vals<S>(a, b, c, d);
    v[q1] = a;
    v[q1 + R] = b;
    v[q1 + 2 * R] = c;
    v[q1 + 3 * R] = d;
  }
}

// Butterflies of pass P >= 1 (radix R = 4 or 2, span Ns) for thread tt: V/R
// butterflies; butterfly m (index j = tt + m T) takes v[m + t (V/R)],
// multiplies by exp(S 2 pi i t (j mod Ns) / (Ns R)) from the per-pass table and
// leaves output q in v[m + q (V/R)].  Pass 0 is the radix-V DFT.
template <int L, int P, int S>
__host__ __device__ __forceinline__ void pass_bfly(float2 (&v)[Passes<L>::V], int tt, const float2* pt) {
  using PS = Passes<L>;
  constexpr int V = PS::V;
  if constexpr (P == 0) {
    dftv<V, S>(v);
  } else {
    constexpr int R = PS::radix(P), Ns = PS::span(P), M = V / R, T = PS::T;
#pragma unroll
    for (int m = 0; m < M; ++m) {
      float2 x[R];
#pragma unroll
      for (int t = 0; t < R; ++t) x[t] = v[m + t * M];
      const int k = (tt + m * T) % Ns;
      const float2* p = pt + PS::twoff(P) + k;
#pragma unroll
      for (int t = 1; t < R; ++t) x[t] = c_mul(x[t], reg::twid<S>(p, (t - 1) * Ns));
      if constexpr (R == V)
        dftv<V, S>(x);
      else
        dft_small<R, S>(x);
#pragma unroll
      for (int q = 0; q < R; ++q) v[m + q * M] = x[q];
    }
  }
}

// Layout of a row group's exchange buffer after the radix-V pass, which
// writes V consecutive elements per thread (lanes V apart, so with the padding
// i + (i >> 4) four or more lanes of a half-warp share a bank pair of the
// 64-bit accesses):
//   1: i ^ ((i >> 2) & 15), an XOR of the four bank bits with bits 2..5 (V = 12,
//      L a multiple of 16: the XOR permutes 16-aligned blocks);
//   2: the padding i + (i >> 2) (V = 20, T = 4, 16, 32): conflict-free writes,
//      two-way stride reads, and addresses that stay base + constant;
//   3: the padding i + (i >> 5) (V = T = 32): writes 32 apart and reads 1
//      apart both conflict-free, addresses base + constant;
//   0: i + (i >> 4) (T = 2, and T = 8 with V = 20, where the others measured
//      slower: their extra address registers spill).
// Counted per half-warp, the exchanges of L = 192 take 112 wavefronts instead
// of 168, of L = 320 224 instead of 304.
__host__ __device__ constexpr int first_layout(int L) {
  return vals_for(L) == 32   ? 3
         : vals_for(L) == 12 ? (L % 16 == 0 ? 1 : 0)
                             : (L / 20 == 4 || L / 20 == 16 || L / 20 == 32 ? 2 : 0);
}

// Position of element i in the exchange buffer after pass P: the layout above
// after pass 0; for V = 12 the XOR with bits 3..6 after pass 1 (L a multiple of
// 16); the padding i + (i >> 4) otherwise.
template <int L, int P>
__host__ __device__ __forceinline__ int xidx(int i) {
  if constexpr (P == 0 && first_layout(L) == 1) {
    return i ^ ((i >> 2) & 15);
  } else if constexpr (P == 0 && first_layout(L) == 2) {
    return i + (i >> 2);
  } else if constexpr (P == 0 && first_layout(L) == 3) {
    return i + (i >> 5);
  } else if constexpr (P == 1 && Passes<L>::V == 12 && L % 16 == 0) {
    return i ^ ((i >> 3) & 15);
  } else {
    return ridx(i);
  }
}

// Stockham writes of pass P: output q of butterfly j goes to o + q Ns with
// o = (j / Ns) Ns R + (j mod Ns).
template <int L, int P>
__host__ __device__ __forceinline__ void pass_store(const float2 (&v)[Passes<L>::V], int tt, float2* out) {
  using PS = Passes<L>;
  constexpr int V = PS::V, R = PS::radix(P), Ns = PS::span(P), M = V / R, T = PS::T;
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const int j = tt + m * T;
    const int o = (j / Ns) * Ns * R + (j % Ns);
#pragma unroll
    for (int q = 0; q < R; ++q) out[xidx<L, P>(o + q * Ns)] = v[m + q * M];
  }
}

// Stride-layout reads after the exchange that follows pass P.
template <int L, int P>
__host__ __device__ __forceinline__ void load_stride(float2 (&v)[Passes<L>::V], int tt, const float2* in) {
  using PS = Passes<L>;
#pragma unroll
  for (int k = 0; k < PS::V; ++k) v[k] = in[xidx<L, P>(tt + k * PS::T)];
}

// Per-pass twiddle table pt[TWSIZE] from tw[m] = exp(-2 pi i m / (L TWSTEP)):
// entry twoff(p) + (t - 1) Ns + k of pass p is exp(-2 pi i t k / (Ns R)).
template <int L, int TWSTEP>
__host__ __device__ __forceinline__ void build_pass_twiddles(float2* pt, const float2* tw, int i0, int stride) {
  using PS = Passes<L>;
  for (int p = 1; p < PS::NPASS; ++p) {
    const int R = PS::radix(p), Ns = PS::span(p), off = PS::twoff(p);
    for (int e = i0; e < (R - 1) * Ns; e += stride) {
      const int t = 1 + e / Ns, k = e % Ns;
      pt[off + e] = tw[t * k * (L / (Ns * R)) * TWSTEP];
    }
  }
}

// Step k (0 .. V/2 - 1) of the in-place inverse packing
// Z[n] = (X_n + conj X_{L-n}) + i e^{+2 pi i n/W} (X_n - conj X_{L-n}): registers
// k and V - 1 - k become Z.  ra, rb are the partner lane's registers V - 1 - k
// and k before this step (unused on lane 0).  Lane 0 pairs registers k and
// V - k; its register V - k was overwritten at step k - 1 and is carried in
// `prev` (X_L before step 0).  tw[m] = exp(-2 pi i m / W).
template <int L>
__host__ __device__ __forceinline__ void pack_step(float2 (&v)[Passes<L>::V], int k, int tt, float2 ra, float2 rb,
                                                   float2& prev, const float2* tw) {
  constexpr int V = Passes<L>::V, T = Passes<L>::T;
  const int k2 = V - 1 - k;
  if (tt == 0) {
    ra = prev;      // X_{L - T k}
    rb = v[k + 1];  // X_{L - T k2}, not yet overwritten
  }
  prev = v[k2];
  const float2 a1 = v[k], a2 = v[k2];
  {
    const float2 c = c_conj(ra);
    v[k] = pack_combine(c_add(a1, c), c_sub(a1, c), tw[tt + k * T]);
  }
  {
    const float2 c = c_conj(rb);
    v[k2] = pack_combine(c_add(a2, c), c_sub(a2, c), tw[tt + k2 * T]);
  }
}

// Forward unpacking X[i] = 1/2 [(Z_i + conj Z_{L-i}) - i e^{-2 pi i i/W} (Z_i - conj Z_{L-i})]
// at i = tt + q T from register q and r, the partner lane's register V - 1 - q
// (on lane 0 Z_{L-i} is its own register (V - q) mod V).  X[L] = Re Z_0 - Im Z_0,
// formed by lane 0.
template <int L>
__host__ __device__ __forceinline__ float2 unpack_value(const float2 (&v)[Passes<L>::V], int q, int tt, float2 r,
                                                        const float2* tw) {
  constexpr int V = Passes<L>::V, T = Passes<L>::T;
  const float2 zb = tt == 0 ? v[q == 0 ? 0 : V - q] : r;
  const float2 c = c_conj(zb);
  return unpack_combine(c_add(v[q], c), c_sub(v[q], c), tw[tt + q * T]);
}

// Exchange buffer of one group (index L included for staging).
__host__ __device__ constexpr int row_buf(int L) {
  return (first_layout(L) == 2 ? L + (L >> 2) : ridx(L)) + 1;  // ridx(L) >= L + (L >> 5)
}

// Batch variants for the column transforms: a CTA transforms KB columns of
// length N; thread (b, tt) holds v[k] = x_b[tt + k T], and element i of column
// b lives at bxidx(i) KB + b of the exchange buffer.  A half-warp spans 16/KB
// values of tt; after the radix-V pass they write V consecutive elements each,
// so i is XORed with bits 2.. of itself (16/KB - 1 of them) to give those
// threads distinct bank pairs; the later exchanges keep the padding.
template <int N, int P, int KB>
__host__ __device__ __forceinline__ int bxidx(int i) {
  if constexpr (P == 0 && N % 4 == 0 && (KB == 8 || KB == 4)) {
    return i ^ ((i >> 2) & (16 / KB - 1));
  } else {
    return ridx(i);
  }
}

template <int N, int P, int KB>
__host__ __device__ __forceinline__ void bpass_store(const float2 (&v)[Passes<N>::V], int tt, int b, float2* out) {
  using PS = Passes<N>;
  constexpr int V = PS::V, R = PS::radix(P), Ns = PS::span(P), M = V / R, T = PS::T;
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const int j = tt + m * T;
    const int o = (j / Ns) * Ns * R + (j % Ns);
#pragma unroll
    for (int q = 0; q < R; ++q) out[bxidx<N, P, KB>(o + q * Ns) * KB + b] = v[m + q * M];
  }
}

template <int N, int P, int KB>
__host__ __device__ __forceinline__ void bload_stride(float2 (&v)[Passes<N>::V], int tt, int b, const float2* in) {
  using PS = Passes<N>;
#pragma unroll
  for (int k = 0; k < PS::V; ++k) v[k] = in[bxidx<N, P, KB>(tt + k * PS::T) * KB + b];
}

// Rows of an exchange buffer of a length-N batch transform.
__host__ __device__ constexpr int brows(int N) { return ridx(N) + 1; }

#ifdef __CUDACC__
// The transform of a CTA's KB columns (every thread of the CTA takes part);
// exchanges alternate between two buffers, so that one CTA barrier per
// exchange suffices (plus one before the first, which also covers the
// previous transform's reads); result in v, stride layout.
template <int N, int S, int KB, int P = 0>
__device__ __forceinline__ void batch_fft(float2 (&v)[Passes<N>::V], int tt, int b, float2* buf0, float2* buf1,
                                          const float2* pt) {
  using PS = Passes<N>;
  pass_bfly<N, P, S>(v, tt, pt);
  if constexpr (P + 1 < PS::NPASS) {
    float2* buf = (P % 2 == 0) ? buf0 : buf1;
    if constexpr (P == 0) __syncthreads();
    bpass_store<N, P, KB>(v, tt, b, buf);
    __syncthreads();
    bload_stride<N, P, KB>(v, tt, b, buf);
    batch_fft<N, S, KB, P + 1>(v, tt, b, buf0, buf1, pt);
  }
}

// The transform of one sequence by its row group (T <= 32: warp barriers);
// result in v, stride layout.  Each exchange starts with a barrier: the buffer
// may still be read by a previous transform.
template <int L, int S, int P = 0>
__device__ __forceinline__ void row_fft(float2 (&v)[Passes<L>::V], int tt, float2* buf, const float2* pt) {
  using PS = Passes<L>;
  pass_bfly<L, P, S>(v, tt, pt);
  if constexpr (P + 1 < PS::NPASS) {
    __syncwarp();
    pass_store<L, P>(v, tt, buf);
    __syncwarp();
    load_stride<L, P>(v, tt, buf);
    row_fft<L, S, P + 1>(v, tt, buf, pt);
  }
}
#endif

}  // namespace rv
}  // namespace shf

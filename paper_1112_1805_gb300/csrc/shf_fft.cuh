// Shared-memory FFT building blocks for sm_103a: mixed-radix (2, 3, 4, 5, 8)
// Stockham stages on float2 data, and the packing that turns a length-W real
// transform into a length-W/2 complex one.  Conventions follow the paper's
// fft2/ifft2 (Sec. 2): forward exponent -1 without scaling, inverse exponent
// +1 (the 1/(H W) factor is applied by the caller).
#pragma once

#include <cuda_runtime.h>

namespace shf {

constexpr int kMaxStages = 16;

// Radix sequence of one transform length L (product of the radices).
struct FftPlan {
  int L;
  int nst;
  int radix[kMaxStages];
};

// Complex sums on the device use the packed FP32x2 adds of sm_100-class GPUs
// (one instruction for both components, IEEE round-to-nearest per component,
// the same values as two scalar adds); the host emulation keeps plain floats.
__host__ __device__ __forceinline__ float2 c_add(float2 a, float2 b) {
#ifdef __CUDA_ARCH__
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
#else
  return make_float2(a.x + b.x, a.y + b.y);
#endif
}
__host__ __device__ __forceinline__ float2 c_sub(float2 a, float2 b) {
#ifdef __CUDA_ARCH__
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
#else
  return make_float2(a.x - b.x, a.y - b.y);
#endif
}
__host__ __device__ __forceinline__ float2 c_mul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// Component-wise a * b and a * b + c: packed FP32x2 multiply and fused
// multiply-add on the device (per component the same IEEE operation as the
// scalar one).
__host__ __device__ __forceinline__ float2 c_mul2(float2 a, float2 b) {
#ifdef __CUDA_ARCH__
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
#else
  return make_float2(a.x * b.x, a.y * b.y);
#endif
}
__host__ __device__ __forceinline__ float2 c_fma2(float2 a, float2 b, float2 c) {
#ifdef __CUDA_ARCH__
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mov.b64 rc, {%6, %7};\n\tfma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
#else
  return make_float2(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y));
#endif
}
// The last step of the real-row packing, s + i conj(w) d with w = e^{-2 pi i k/W}
// (i conj w = (w.y, w.x): one complex product and one packed add).
__host__ __device__ __forceinline__ float2 pack_combine(float2 s, float2 d, float2 w) {
  return c_add(s, c_mul(make_float2(w.y, w.x), d));
}
// The last step of the real-row unpacking, (s - i w d) / 2 (-i w = (w.y, -w.x)).
__host__ __device__ __forceinline__ float2 unpack_combine(float2 s, float2 d, float2 w) {
  return c_mul2(c_add(s, c_mul(make_float2(w.y, -w.x), d)), make_float2(0.5f, 0.5f));
}
__host__ __device__ __forceinline__ float2 c_conj(float2 a) { return make_float2(a.x, -a.y); }
__host__ __device__ __forceinline__ float2 c_scale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// a * (S i) for S = +1 or -1
template <int S>
__host__ __device__ __forceinline__ float2 c_mul_si(float2 a) {
  return make_float2(-static_cast<float>(S) * a.y, static_cast<float>(S) * a.x);
}

// In-place R-point DFTs V_q = sum_t v_t exp(S 2 pi i t q / R).
template <int S>
__host__ __device__ __forceinline__ void dft2(float2* v) {
  const float2 t = c_sub(v[0], v[1]);
  v[0] = c_add(v[0], v[1]);
  v[1] = t;
}

template <int S>
__host__ __device__ __forceinline__ void dft4_vals(float2& a0, float2& a1, float2& a2, float2& a3) {
  const float2 s02 = c_add(a0, a2), d02 = c_sub(a0, a2);
  const float2 s13 = c_add(a1, a3), t = c_sub(a1, a3);
  a0 = c_add(s02, s13);
  a2 = c_sub(s02, s13);
  // d02 +- S i t with the swapped components in scalar adds (a packed add
  // would first have to move them into a register pair)
  const float s = static_cast<float>(S);
  a1 = make_float2(d02.x - s * t.y, d02.y + s * t.x);
  a3 = make_float2(d02.x + s * t.y, d02.y - s * t.x);
}

template <int S>
__host__ __device__ __forceinline__ void dft4(float2* v) {
  dft4_vals<S>(v[0], v[1], v[2], v[3]);
}

template <int S>
__host__ __device__ __forceinline__ void dft8(float2* v) {
  float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4_vals<S>(e0, e1, e2, e3);
  dft4_vals<S>(o0, o1, o2, o3);
  const float r = 0.70710678118654752440f;
  const float s = static_cast<float>(S);
  const float2 t1 = make_float2(r * (o1.x - s * o1.y), r * (o1.y + s * o1.x));    // * (1 + S i)/sqrt(2)
  const float2 t2 = c_mul_si<S>(o2);                                               // * S i
  const float2 t3 = make_float2(r * (-o3.x - s * o3.y), r * (-o3.y + s * o3.x));  // * (-1 + S i)/sqrt(2)
  v[0] = c_add(e0, o0);
  v[4] = c_sub(e0, o0);
  v[1] = c_add(e1, t1);
  v[5] = c_sub(e1, t1);
  v[2] = c_add(e2, t2);
  v[6] = c_sub(e2, t2);
  v[3] = c_add(e3, t3);
  v[7] = c_sub(e3, t3);
}

template <int S>
__host__ __device__ __forceinline__ void dft3(float2* v) {
  const float h = static_cast<float>(S) * 0.86602540378443864676f;  // S sin(2 pi / 3)
  const float2 t1 = c_add(v[1], v[2]), t2 = c_sub(v[1], v[2]);
  const float2 m = make_float2(v[0].x - 0.5f * t1.x, v[0].y - 0.5f * t1.y);
  const float2 n = make_float2(-h * t2.y, h * t2.x);
  v[0] = c_add(v[0], t1);
  v[1] = c_add(m, n);
  v[2] = c_sub(m, n);
}

template <int S>
__host__ __device__ __forceinline__ void dft5(float2* v) {
  const float c1 = 0.30901699437494742410f, c2 = -0.80901699437494742410f;  // cos(2pi/5), cos(4pi/5)
  const float s1 = static_cast<float>(S) * 0.95105651629515357212f;         // S sin(2pi/5)
  const float s2 = static_cast<float>(S) * 0.58778525229247312917f;         // S sin(4pi/5)
  const float2 a1 = c_add(v[1], v[4]), b1 = c_sub(v[1], v[4]);
  const float2 a2 = c_add(v[2], v[3]), b2 = c_sub(v[2], v[3]);
  const float2 p1 = make_float2(v[0].x + c1 * a1.x + c2 * a2.x, v[0].y + c1 * a1.y + c2 * a2.y);
  const float2 p2 = make_float2(v[0].x + c2 * a1.x + c1 * a2.x, v[0].y + c2 * a1.y + c1 * a2.y);
  const float2 r1 = make_float2(s1 * b1.x + s2 * b2.x, s1 * b1.y + s2 * b2.y);
  const float2 r2 = make_float2(s2 * b1.x - s1 * b2.x, s2 * b1.y - s1 * b2.y);
  const float2 q1 = make_float2(-r1.y, r1.x);  // i * r1 (S folded into s1, s2)
  const float2 q2 = make_float2(-r2.y, r2.x);
  v[0] = make_float2(v[0].x + a1.x + a2.x, v[0].y + a1.y + a2.y);
  v[1] = c_add(p1, q1);
  v[4] = c_sub(p1, q1);
  v[2] = c_add(p2, q2);
  v[3] = c_sub(p2, q2);
}

template <int R, int S>
__host__ __device__ __forceinline__ void dft_small(float2* v) {
  if (R == 2) dft2<S>(v);
  if (R == 3) dft3<S>(v);
  if (R == 4) dft4<S>(v);
  if (R == 5) dft5<S>(v);
  if (R == 8) dft8<S>(v);
}

// One butterfly of a Stockham stage of length L, radix R, sub-transform span
// Ns (product of the radices of the earlier stages).  Element (i, b) of the
// batch lives at ptr[i*istride + b*bstride].  Reads in(j + t L/R), applies
// the twiddles exp(S 2 pi i t (j mod Ns) / (Ns R)), an R-point DFT, and writes
// out((j / Ns) Ns R + (j mod Ns) + q Ns).  tw[m] = exp(-2 pi i m / (L twstep)).
template <int R, int S>
__host__ __device__ __forceinline__ void stockham_bfly(const float2* in, float2* out, int L, int Ns, int j, int b,
                                                       int istride, int bstride, const float2* tw, int twstep) {
  const int nb = L / R;
  float2 v[R];
#pragma unroll
  for (int t = 0; t < R; ++t) v[t] = in[(j + t * nb) * istride + b * bstride];
  const int k = j % Ns;
  if (Ns > 1) {
    const int base = k * (L / (Ns * R)) * twstep;
#pragma unroll
    for (int t = 1; t < R; ++t) {
      float2 w = tw[t * base];
      if (S > 0) w.y = -w.y;
      v[t] = c_mul(v[t], w);
    }
  }
  dft_small<R, S>(v);
  const int o = (j / Ns) * Ns * R + k;
#pragma unroll
  for (int q = 0; q < R; ++q) out[(o + q * Ns) * istride + b * bstride] = v[q];
}

// Work item `idx` of a stage: BATCH_FAST maps consecutive items to
// consecutive batch members (column transforms of a row-major tile),
// otherwise to consecutive butterflies of one sequence (row transforms).
template <int S, bool BATCH_FAST>
__host__ __device__ __forceinline__ void stockham_item(const float2* in, float2* out, int L, int R, int Ns, int idx,
                                                       int B, int istride, int bstride, const float2* tw,
                                                       int twstep) {
  const int nb = L / R;
  int j, b;
  if (BATCH_FAST) {
    b = idx % B;
    j = idx / B;
  } else {
    j = idx % nb;
    b = idx / nb;
  }
  switch (R) {
    case 2: stockham_bfly<2, S>(in, out, L, Ns, j, b, istride, bstride, tw, twstep); break;
    case 3: stockham_bfly<3, S>(in, out, L, Ns, j, b, istride, bstride, tw, twstep); break;
    case 4: stockham_bfly<4, S>(in, out, L, Ns, j, b, istride, bstride, tw, twstep); break;
    case 5: stockham_bfly<5, S>(in, out, L, Ns, j, b, istride, bstride, tw, twstep); break;
    default: stockham_bfly<8, S>(in, out, L, Ns, j, b, istride, bstride, tw, twstep); break;
  }
}

#ifdef __CUDACC__
// A batch of B transforms of length p.L in shared memory, ping-ponging
// between a and b; returns the buffer holding the natural-order result.
// All threads of the block must call it (it synchronises after each stage).
template <int S, bool BATCH_FAST>
__device__ __forceinline__ float2* stockham(float2* a, float2* b, const FftPlan& p, int B, int istride, int bstride,
                                            const float2* __restrict__ tw, int twstep) {
  int Ns = 1;
  for (int s = 0; s < p.nst; ++s) {
    const int R = p.radix[s];
    const int total = (p.L / R) * B;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x)
      stockham_item<S, BATCH_FAST>(a, b, p.L, R, Ns, idx, B, istride, bstride, tw, twstep);
    __syncthreads();
    float2* t = a;
    a = b;
    b = t;
    Ns *= R;
  }
  return a;
}
#endif

// Real transforms of length W = 2L through one complex transform of length L.
// twW[m] = exp(-2 pi i m / W).
//
// Inverse packing: from the half spectrum X[0..L] of a real row, the complex
// sequence whose unscaled inverse DFT of length L has the even samples of the
// unscaled length-W inverse in its real part and the odd samples in its
// imaginary part:  Z[k] = (X[k] + conj X[L-k]) + i e^{+2 pi i k/W} (X[k] - conj X[L-k]).
__host__ __device__ __forceinline__ float2 c2r_pack(const float2* X, int L, int k, const float2* twW) {
  const float2 a = X[k];
  const float2 b = c_conj(X[L - k]);
  const float2 s = c_add(a, b), d = c_sub(a, b);
  return pack_combine(s, d, twW[k]);
}

// Forward unpacking: Z = DFT_L(x[2n] + i x[2n+1]); returns X[k], k = 0..L,
// X[k] = 1/2 [ (Z_k + conj Z_{L-k}) - i e^{-2 pi i k/W} (Z_k - conj Z_{L-k}) ] (indices mod L).
__host__ __device__ __forceinline__ float2 r2c_unpack(const float2* Z, int L, int k, const float2* twW) {
  const float2 a = Z[k == L ? 0 : k];
  const float2 b = c_conj(Z[k == 0 ? 0 : L - k]);
  const float2 s = c_add(a, b), d = c_sub(a, b);
  return unpack_combine(s, d, twW[k]);
}

// Radix sequence for L = 2^a 3^b 5^c (8s first, then a 4 or 2, then 3s and
// 5s); returns false when L has another prime factor or too many stages.
inline bool make_plan(int L, FftPlan* p) {
  p->L = L;
  p->nst = 0;
  int n = L, a = 0;
  while (n % 2 == 0) {
    n /= 2;
    ++a;
  }
  int b = 0, c = 0;
  while (n % 3 == 0) {
    n /= 3;
    ++b;
  }
  while (n % 5 == 0) {
    n /= 5;
    ++c;
  }
  if (n != 1 || L < 1) return false;
  auto push = [&](int r) {
    if (p->nst >= kMaxStages) return false;
    p->radix[p->nst++] = r;
    return true;
  };
  for (int i = 0; i < a / 3; ++i)
    if (!push(8)) return false;
  if (a % 3 == 2 && !push(4)) return false;
  if (a % 3 == 1 && !push(2)) return false;
  for (int i = 0; i < b; ++i)
    if (!push(3)) return false;
  for (int i = 0; i < c; ++i)
    if (!push(5)) return false;
  return true;
}

}  // namespace shf

// Fast path for power-of-two sizes (8 <= H <= 1024, 16 <= W <= 2048): the
// per-filter work of an ADMM iteration (Sec. 3 of Haeuser & Steidl) with
// register-resident FFTs (shf_fft_reg.cuh).
//
// One iteration, after the u/w-step (k_row_ustep) has left the row spectra of
// u in Ur:
//   k_fcol_fwd      Ur -> Uhat, the full 2-D spectrum of u, once per label;
//   per label k, per wave of filters [f0, f0 + nf):
//     k_fcol_fan      Y_f = column-inverse(W_f * Uhat_k) for f in the wave
//     k_frow_shrink   row-inverse, g = b_v + S u, b_v <- clip(g), d = soft(g) -
//                     clip(g) (= v - b_v), row-forward of d, in place in Y_f
//     k_fcol_gather   partial_g += sum_{f in group g} W_f * column-forward(Y_f)
//   k_fcol_reduce_inv  T_k = column-inverse(sum_g partial_g)
// The coefficient spectra of one wave (a few tens of MB) stay in L2 between
// the three kernels; b_v is streamed with evict-first hints.
#include <algorithm>

#include "shf_fft_reg.cuh"
#include "shf_internal.h"

namespace shf {

namespace {

using reg::kB;
using reg::kS;
using reg::sidx;

__device__ __forceinline__ void load_table(float2* dst, const float2* __restrict__ src, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

// ---------------------------------------------------------------------------
// Column kernels: a CTA of H threads owns 8 consecutive half-spectrum columns
// (thread (b, tt) holds rows tt + k H/8 of column 8*blockIdx.x + b).
// ---------------------------------------------------------------------------

template <int H>
__global__ void __launch_bounds__(H) k_fcol_fwd(const float2* __restrict__ in, float2* __restrict__ out, int Wh,
                                                const float2* __restrict__ twH) {
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* b0 = sm + H;
  float2* b1 = b0 + H * kS;
  load_table(tw, twH, H);
  __syncthreads();
  const int b = threadIdx.x & 7, tt = threadIdx.x >> 3;
  const int col = blockIdx.x * kB + b;
  const bool ok = col < Wh;
  const size_t plane = static_cast<size_t>(H) * Wh * blockIdx.y;
  float2 v[8];
#pragma unroll
  for (int k = 0; k < 8; ++k)
    v[k] = ok ? in[plane + static_cast<size_t>(tt + k * (H / 8)) * Wh + col] : make_float2(0.f, 0.f);
  reg::fft<H, -1, 1>(v, tt, b, b0, b1, tw);
  if (ok) {
#pragma unroll
    for (int k = 0; k < 8; ++k) out[plane + static_cast<size_t>(tt + k * (H / 8)) * Wh + col] = v[k];
  }
}

template <int H>
__global__ void __launch_bounds__(H) k_fcol_fan(const float2* __restrict__ uhat, const float* __restrict__ bank,
                                                float2* __restrict__ Y, int Wh, int label, int f0, int nf, int fg,
                                                const float2* __restrict__ twH) {
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* b0 = sm + H;
  float2* b1 = b0 + H * kS;
  load_table(tw, twH, H);
  __syncthreads();
  const int b = threadIdx.x & 7, tt = threadIdx.x >> 3;
  const int col = blockIdx.x * kB + b;
  const bool ok = col < Wh;
  const size_t P = static_cast<size_t>(H) * Wh;
  float2 u[8];
#pragma unroll
  for (int k = 0; k < 8; ++k)
    u[k] = ok ? uhat[P * label + static_cast<size_t>(tt + k * (H / 8)) * Wh + col] : make_float2(0.f, 0.f);
  const int fb = blockIdx.y * fg, fe = min(nf, fb + fg);
  for (int fl = fb; fl < fe; ++fl) {
    const float* wf = bank + P * (f0 + fl);
    float2 v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const float w = ok ? __ldg(wf + static_cast<size_t>(tt + k * (H / 8)) * Wh + col) : 0.f;
      v[k] = c_scale(u[k], w);
    }
    reg::fft<H, +1, 1>(v, tt, b, b0, b1, tw);
    if (ok) {
      float2* dst = Y + P * fl;
#pragma unroll
      for (int k = 0; k < 8; ++k) dst[static_cast<size_t>(tt + k * (H / 8)) * Wh + col] = v[k];
    }
  }
}

// partial[g][label] (+)= sum over the group's filters of W_f * column-forward(Y_f);
// accumulate != 0 adds to what an earlier wave left there.
template <int H>
__global__ void __launch_bounds__(H) k_fcol_gather(const float2* __restrict__ Y, const float* __restrict__ bank,
                                                   float2* __restrict__ partial, int Wh, int K, int label, int f0,
                                                   int nf, int fg, int accumulate, const float2* __restrict__ twH) {
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* b0 = sm + H;
  float2* b1 = b0 + H * kS;
  load_table(tw, twH, H);
  __syncthreads();
  const int b = threadIdx.x & 7, tt = threadIdx.x >> 3;
  const int col = blockIdx.x * kB + b;
  const bool ok = col < Wh;
  const size_t P = static_cast<size_t>(H) * Wh;
  float2 acc[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) acc[k] = make_float2(0.f, 0.f);
  const int fb = blockIdx.y * fg, fe = min(nf, fb + fg);
  for (int fl = fb; fl < fe; ++fl) {
    const float2* src = Y + P * fl;
    float2 v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k)
      v[k] = ok ? src[static_cast<size_t>(tt + k * (H / 8)) * Wh + col] : make_float2(0.f, 0.f);
    reg::fft<H, -1, 1>(v, tt, b, b0, b1, tw);
    const float* wf = bank + P * (f0 + fl);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const float w = ok ? __ldg(wf + static_cast<size_t>(tt + k * (H / 8)) * Wh + col) : 0.f;
      acc[k].x = fmaf(w, v[k].x, acc[k].x);
      acc[k].y = fmaf(w, v[k].y, acc[k].y);
    }
  }
  if (ok) {
    float2* dst = partial + P * (static_cast<size_t>(blockIdx.y) * K + label);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const size_t off = static_cast<size_t>(tt + k * (H / 8)) * Wh + col;
      dst[off] = accumulate ? c_add(dst[off], acc[k]) : acc[k];
    }
  }
}

template <int H>
__global__ void __launch_bounds__(H) k_fcol_reduce_inv(const float2* __restrict__ partial, float2* __restrict__ T,
                                                       int Wh, int K, int groups, const float2* __restrict__ twH) {
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* b0 = sm + H;
  float2* b1 = b0 + H * kS;
  load_table(tw, twH, H);
  __syncthreads();
  const int b = threadIdx.x & 7, tt = threadIdx.x >> 3;
  const int col = blockIdx.x * kB + b;
  const bool ok = col < Wh;
  const size_t P = static_cast<size_t>(H) * Wh;
  const int label = blockIdx.y;
  float2 v[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = make_float2(0.f, 0.f);
  if (ok) {
    for (int g = 0; g < groups; ++g) {  // fixed order over the groups
      const float2* src = partial + P * (static_cast<size_t>(g) * K + label) + col;
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = c_add(v[k], src[static_cast<size_t>(tt + k * (H / 8)) * Wh]);
    }
  }
  reg::fft<H, +1, 1>(v, tt, b, b0, b1, tw);
  if (ok) {
#pragma unroll
    for (int k = 0; k < 8; ++k) T[P * label + static_cast<size_t>(tt + k * (H / 8)) * Wh + col] = v[k];
  }
}

// ---------------------------------------------------------------------------
// Row kernel: a CTA of L threads owns 8 consecutive rows of one coefficient
// plane; a real row of length W = 2L is the complex row z[n] = x[2n] + i x[2n+1].
// ---------------------------------------------------------------------------

// v-step and b_v update of Sec. 3 on rows of (S u)_f: g = b_v + c,
// b_v <- clip(g, -t, t), d = soft(g, t) - clip(g, -t, t) = g - 2 clip(g);
// d (= v - b_v of the new iterate) is transformed back in place.
template <int L>
__global__ void __launch_bounds__(L) k_frow_shrink(float2* __restrict__ Y, float* __restrict__ bv,
                                                   const float* __restrict__ thr, int H, int eta, int label, int f0,
                                                   float scale, const float2* __restrict__ twW) {
  constexpr int Wh = L + 1;
  extern __shared__ float2 sm[];
  float2* tw = sm;                 // 2L entries: exp(-2 pi i m / W)
  float2* b0 = sm + 2 * L;         // L * kS
  float2* b1 = b0 + L * kS;        // (L + 1) * kS, also the staging buffer
  load_table(tw, twW, 2 * L);
  const int row0 = blockIdx.x * kB;
  const int fl = blockIdx.y;
  float2* X = Y + static_cast<size_t>(H) * Wh * fl;
  // stage the 8 half-spectrum rows, index-fast (coalesced, conflict-free)
  for (int e = threadIdx.x; e < kB * Wh; e += L) {
    const int r = e / Wh, i = e - r * Wh, row = row0 + r;
    b1[sidx(i, r)] = row < H ? X[static_cast<size_t>(row) * Wh + i] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const int b = threadIdx.x & 7, tt = threadIdx.x >> 3;
  float2 v[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {  // inverse packing Z[n] = (X_n + conj X_{L-n}) + i e^{+2 pi i n/W} (X_n - conj X_{L-n})
    const int n = tt + k * (L / 8);
    const float2 a = b1[sidx(n, b)];
    const float2 c = c_conj(b1[sidx(L - n, b)]);
    const float2 s = c_add(a, c), d = c_sub(a, c);
    const float2 t = c_mul(c_conj(tw[n]), d);
    v[k] = make_float2(s.x - t.y, s.y + t.x);
  }
  reg::fft<L, +1, 2>(v, tt, b, b0, b1, tw);
  const int row = row0 + b;
  const int f = f0 + fl;
  const float th = thr[f];
  if (row < H) {
    float2* b2 = reinterpret_cast<float2*>(bv) + (static_cast<size_t>(label) * eta + f) * H * L +
                 static_cast<size_t>(row) * L;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int n = tt + k * (L / 8);
      const float2 bo = __ldcs(b2 + n);
      const float gx = fmaf(scale, v[k].x, bo.x), gy = fmaf(scale, v[k].y, bo.y);
      const float cx = fminf(fmaxf(gx, -th), th), cy = fminf(fmaxf(gy, -th), th);
      __stcs(b2 + n, make_float2(cx, cy));
      v[k] = make_float2(gx - 2.f * cx, gy - 2.f * cy);
    }
  } else {
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = make_float2(0.f, 0.f);
  }
  reg::fft<L, -1, 2>(v, tt, b, b0, b1, tw);
  __syncthreads();  // the last pass may still read b1
#pragma unroll
  for (int k = 0; k < 8; ++k) b1[sidx(tt + k * (L / 8), b)] = v[k];
  __syncthreads();
  // forward unpacking X[k] = 1/2 [(Z_k + conj Z_{L-k}) - i e^{-2 pi i k/W} (Z_k - conj Z_{L-k})]
  for (int e = threadIdx.x; e < kB * Wh; e += L) {
    const int r = e / Wh, i = e - r * Wh, rw = row0 + r;
    if (rw < H) {
      const float2 a = b1[sidx(i == L ? 0 : i, r)];
      const float2 c = c_conj(b1[sidx(i == 0 ? 0 : L - i, r)]);
      const float2 s = c_add(a, c), d = c_sub(a, c);
      const float2 t = c_mul(tw[i], d);
      X[static_cast<size_t>(rw) * Wh + i] = make_float2(0.5f * (s.x + t.y), 0.5f * (s.y - t.x));
    }
  }
}

template <int N>
size_t col_smem() {
  return sizeof(float2) * (N + 2 * N * kS);
}

template <int L>
size_t row_smem() {
  return sizeof(float2) * (2 * L + L * kS + (L + 1) * kS);
}

int groups_for(const Geo& g, int nf) {
  // enough CTAs for about two per SM, at least two filters per group
  const int want = (2 * 152 + g.ntiles - 1) / g.ntiles;
  int fg = (nf + want - 1) / want;
  if (fg < 2) fg = 2;
  if (fg > nf) fg = nf;
  return fg;
}

// One filter-group size for every wave, so that later waves never use a group
// the first wave of the label did not initialise.
template <int H, int L>
cudaError_t per_filter_waves(const Geo& g, const float2* uhat, float2* Y, float* bv, const float* thr,
                             float2* partial, int K, int wave, float scale, cudaStream_t st, const LaunchHook& hook,
                             int* groups_out) {
  const int ntiles = (g.Wh + kB - 1) / kB;
  const int fg = groups_for(g, wave);
  int groups = 0;
  for (int label = 0; label < K; ++label) {
    for (int f0 = 0; f0 < g.eta; f0 += wave) {
      const int nf = min(wave, g.eta - f0);
      const int ng = (nf + fg - 1) / fg;
      hook.mark(kKindFan);
      k_fcol_fan<H><<<dim3(ntiles, ng), H, col_smem<H>(), st>>>(uhat, g.bank, Y, g.Wh, label, f0, nf, fg, g.twH);
      hook.mark(kKindShrink);
      k_frow_shrink<L><<<dim3((g.H + kB - 1) / kB, nf), L, row_smem<L>(), st>>>(Y, bv, thr, g.H, g.eta, label, f0,
                                                                                scale, g.twW);
      hook.mark(kKindGather);
      k_fcol_gather<H><<<dim3(ntiles, ng), H, col_smem<H>(), st>>>(Y, g.bank, partial, g.Wh, K, label, f0, nf, fg,
                                                                   f0 > 0 ? 1 : 0, g.twH);
      if (ng > groups) groups = ng;
    }
  }
  *groups_out = groups;
  return cudaGetLastError();
}

template <int H, int L>
cudaError_t iteration_body(const Geo& g, const float2* Ur, float2* uhat, float2* Y, float* bv, const float* thr,
                           float2* partial, float2* T, int K, int wave, float scale, cudaStream_t st,
                           const LaunchHook& hook) {
  const int ntiles = (g.Wh + kB - 1) / kB;
  hook.mark(kKindColFwd);
  k_fcol_fwd<H><<<dim3(ntiles, K), H, col_smem<H>(), st>>>(Ur, uhat, g.Wh, g.twH);
  int groups = 0;
  cudaError_t e = per_filter_waves<H, L>(g, uhat, Y, bv, thr, partial, K, wave, scale, st, hook, &groups);
  if (e != cudaSuccess) return e;
  hook.mark(kKindReduce);
  k_fcol_reduce_inv<H><<<dim3(ntiles, K), H, col_smem<H>(), st>>>(partial, T, g.Wh, K, groups, g.twH);
  return cudaGetLastError();
}

template <typename KERN>
cudaError_t allow_smem(KERN k, size_t bytes) {
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes));
}

template <int H>
cudaError_t prepare_col() {
  const size_t s = col_smem<H>();
  cudaError_t e = allow_smem(k_fcol_fwd<H>, s);
  if (e == cudaSuccess) e = allow_smem(k_fcol_fan<H>, s);
  if (e == cudaSuccess) e = allow_smem(k_fcol_gather<H>, s);
  if (e == cudaSuccess) e = allow_smem(k_fcol_reduce_inv<H>, s);
  return e;
}

template <int L>
cudaError_t prepare_row() {
  return allow_smem(k_frow_shrink<L>, row_smem<L>());
}

template <int H>
cudaError_t dispatch_L(const Geo& g, const float2* Ur, float2* uhat, float2* Y, float* bv, const float* thr,
                       float2* partial, float2* T, int K, int wave, float scale, cudaStream_t st,
                       const LaunchHook& hook) {
  switch (g.L) {
    case 8: return iteration_body<H, 8>(g, Ur, uhat, Y, bv, thr, partial, T, K, wave, scale, st, hook);
    case 16: return iteration_body<H, 16>(g, Ur, uhat, Y, bv, thr, partial, T, K, wave, scale, st, hook);
    case 32: return iteration_body<H, 32>(g, Ur, uhat, Y, bv, thr, partial, T, K, wave, scale, st, hook);
    case 64: return iteration_body<H, 64>(g, Ur, uhat, Y, bv, thr, partial, T, K, wave, scale, st, hook);
    case 128: return iteration_body<H, 128>(g, Ur, uhat, Y, bv, thr, partial, T, K, wave, scale, st, hook);
    case 256: return iteration_body<H, 256>(g, Ur, uhat, Y, bv, thr, partial, T, K, wave, scale, st, hook);
    case 512: return iteration_body<H, 512>(g, Ur, uhat, Y, bv, thr, partial, T, K, wave, scale, st, hook);
    case 1024: return iteration_body<H, 1024>(g, Ur, uhat, Y, bv, thr, partial, T, K, wave, scale, st, hook);
    default: return cudaErrorInvalidValue;
  }
}

bool pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

}  // namespace

bool fast_path_ok(const Geo& g) {
  return pow2(g.H) && pow2(g.L) && g.H >= 8 && g.H <= 1024 && g.L >= 8 && g.L <= 1024;
}

cudaError_t prepare_fast_kernels() {
  const cudaError_t errs[] = {prepare_col<8>(),   prepare_col<16>(),  prepare_col<32>(),  prepare_col<64>(),
                              prepare_col<128>(), prepare_col<256>(), prepare_col<512>(), prepare_col<1024>(),
                              prepare_row<8>(),   prepare_row<16>(),  prepare_row<32>(),  prepare_row<64>(),
                              prepare_row<128>(), prepare_row<256>(), prepare_row<512>(), prepare_row<1024>()};
  for (cudaError_t e : errs)
    if (e != cudaSuccess) return e;
  return cudaSuccess;
}

int fast_wave(const Geo& g) {
  // filters per wave: keep the wave's coefficient spectra near 32 MiB
  const size_t plane = sizeof(float2) * static_cast<size_t>(g.H) * g.Wh;
  int w = static_cast<int>((size_t(32) << 20) / plane);
  if (w < 1) w = 1;
  if (w > g.eta) w = g.eta;
  // balance the waves of a label
  const int nw = (g.eta + w - 1) / w;
  return (g.eta + nw - 1) / nw;
}

int fast_groups_max(const Geo& g) {
  const int wave = fast_wave(g);
  const int fg = groups_for(g, wave);
  return (wave + fg - 1) / fg;
}

cudaError_t run_fast_iteration_body(const Geo& g, const float2* Ur, float2* uhat, float2* Y, float* bv,
                                    const float* thr, float2* partial, float2* T, int K, float scale,
                                    cudaStream_t st, const LaunchHook& hook) {
  const int wave = fast_wave(g);
  switch (g.H) {
    case 8: return dispatch_L<8>(g, Ur, uhat, Y, bv, thr, partial, T, K, wave, scale, st, hook);
    case 16: return dispatch_L<16>(g, Ur, uhat, Y, bv, thr, partial, T, K, wave, scale, st, hook);
    case 32: return dispatch_L<32>(g, Ur, uhat, Y, bv, thr, partial, T, K, wave, scale, st, hook);
    case 64: return dispatch_L<64>(g, Ur, uhat, Y, bv, thr, partial, T, K, wave, scale, st, hook);
    case 128: return dispatch_L<128>(g, Ur, uhat, Y, bv, thr, partial, T, K, wave, scale, st, hook);
    case 256: return dispatch_L<256>(g, Ur, uhat, Y, bv, thr, partial, T, K, wave, scale, st, hook);
    case 512: return dispatch_L<512>(g, Ur, uhat, Y, bv, thr, partial, T, K, wave, scale, st, hook);
    case 1024: return dispatch_L<1024>(g, Ur, uhat, Y, bv, thr, partial, T, K, wave, scale, st, hook);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace shf

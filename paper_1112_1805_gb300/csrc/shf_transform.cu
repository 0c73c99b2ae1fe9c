// Shearlet transform and ADMM kernels (Haeuser & Steidl, arXiv:1112.1805).
//
// A 2-D transform of an H x W real plane is split into row transforms (real
// length W, packed into complex length W/2) and column transforms (complex
// length H) over the W/2+1 columns of the half spectrum.  The filters are real
// and even, so every product of a filter with the spectrum of a real plane is
// again the half spectrum of a real plane.
//
// Analysis S (eq. wichtig), for each channel:
//   row-forward -> [k_col_fan: column-forward, then per filter f:
//                   multiply by W_f, column-inverse] -> row-inverse.
// Synthesis S^T (Fourier-domain form after the Theorem), for each channel:
//   row-forward of every coefficient plane -> [k_col_gather: column-forward,
//   multiply by W_f, sum over a filter group] -> [k_col_reduce_inv: sum over
//   groups in fixed order, column-inverse] -> row-inverse.
// ADMM iteration (Sec. 3), state (b_v, T = column-inverse of the synthesis
// spectrum of v - b_v, w, b_w):
//   k_row_ustep   : T -> S^T(v-b_v); u-step; w-step; b_w; row-forward of u
//   k_col_fan     : u spectra -> per-filter coefficient spectra
//   k_row_shrink  : row-inverse -> g = b_v + Su; b_v <- clip(g); d = soft(g) - clip(g)
//                   = v - b_v; row-forward of d (in place)
//   k_col_gather + k_col_reduce_inv : synthesis spectrum of d -> T
#include <algorithm>

#include "shf_internal.h"
#include "shf_simplex.cuh"

namespace shf {

namespace {

// ---------------------------------------------------------------------------
// Column kernels: one CTA owns a tile of TC consecutive half-spectrum columns
// over all H rows, stored row-major [H][TC] in shared memory (coalesced
// loads; consecutive threads work on consecutive columns).
// ---------------------------------------------------------------------------

template <int MAXE>
__global__ void __launch_bounds__(kColThreads)
    k_col_fan(const float2* __restrict__ in, const float* __restrict__ bank, float2* __restrict__ out, int H, int Wh,
              int eta, int TC, int fg, FftPlan pH, const float2* __restrict__ twH) {
  extern __shared__ float2 sm[];
  const int E = H * TC;
  float2* A = sm;
  float2* B = sm + E;
  const int col0 = blockIdx.x * TC, ch = blockIdx.y;
  const int f_begin = blockIdx.z * fg, f_end = min(eta, f_begin + fg);
  const float2* src = in + static_cast<size_t>(ch) * H * Wh;
  for (int e = threadIdx.x; e < E; e += kColThreads) {
    const int r = e / TC, col = col0 + (e - r * TC);
    A[e] = col < Wh ? src[static_cast<size_t>(r) * Wh + col] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const float2* U = stockham<-1, true>(A, B, pH, TC, TC, 1, twH, 1);
  float2 uh[MAXE];
#pragma unroll
  for (int m = 0; m < MAXE; ++m) {
    const int e = threadIdx.x + m * kColThreads;
    uh[m] = e < E ? U[e] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  for (int f = f_begin; f < f_end; ++f) {
    const float* wf = bank + static_cast<size_t>(f) * H * Wh;
#pragma unroll
    for (int m = 0; m < MAXE; ++m) {
      const int e = threadIdx.x + m * kColThreads;
      if (e < E) {
        const int r = e / TC, col = col0 + (e - r * TC);
        const float w = col < Wh ? __ldg(wf + static_cast<size_t>(r) * Wh + col) : 0.f;
        A[e] = c_scale(uh[m], w);
      }
    }
    __syncthreads();
    const float2* Y = stockham<+1, true>(A, B, pH, TC, TC, 1, twH, 1);
    float2* dst = out + (static_cast<size_t>(ch) * eta + f) * H * Wh;
    for (int e = threadIdx.x; e < E; e += kColThreads) {
      const int r = e / TC, col = col0 + (e - r * TC);
      if (col < Wh) dst[static_cast<size_t>(r) * Wh + col] = Y[e];
    }
    __syncthreads();
  }
}

template <int MAXE>
__global__ void __launch_bounds__(kColThreads)
    k_col_gather(const float2* __restrict__ in, const float* __restrict__ bank, float2* __restrict__ partial, int H,
                 int Wh, int eta, int nch, int TC, int fg, FftPlan pH, const float2* __restrict__ twH) {
  extern __shared__ float2 sm[];
  const int E = H * TC;
  float2* A = sm;
  float2* B = sm + E;
  const int col0 = blockIdx.x * TC, ch = blockIdx.y, grp = blockIdx.z;
  const int f_begin = grp * fg, f_end = min(eta, f_begin + fg);
  float2 acc[MAXE];
#pragma unroll
  for (int m = 0; m < MAXE; ++m) acc[m] = make_float2(0.f, 0.f);
  for (int f = f_begin; f < f_end; ++f) {
    const float2* src = in + (static_cast<size_t>(ch) * eta + f) * H * Wh;
    for (int e = threadIdx.x; e < E; e += kColThreads) {
      const int r = e / TC, col = col0 + (e - r * TC);
      A[e] = col < Wh ? src[static_cast<size_t>(r) * Wh + col] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const float2* Z = stockham<-1, true>(A, B, pH, TC, TC, 1, twH, 1);
    const float* wf = bank + static_cast<size_t>(f) * H * Wh;
#pragma unroll
    for (int m = 0; m < MAXE; ++m) {
      const int e = threadIdx.x + m * kColThreads;
      if (e < E) {
        const int r = e / TC, col = col0 + (e - r * TC);
        const float w = col < Wh ? __ldg(wf + static_cast<size_t>(r) * Wh + col) : 0.f;
        acc[m].x = fmaf(w, Z[e].x, acc[m].x);
        acc[m].y = fmaf(w, Z[e].y, acc[m].y);
      }
    }
    __syncthreads();
  }
  float2* dst = partial + (static_cast<size_t>(grp) * nch + ch) * H * Wh;
#pragma unroll
  for (int m = 0; m < MAXE; ++m) {
    const int e = threadIdx.x + m * kColThreads;
    if (e < E) {
      const int r = e / TC, col = col0 + (e - r * TC);
      if (col < Wh) dst[static_cast<size_t>(r) * Wh + col] = acc[m];
    }
  }
}

__global__ void __launch_bounds__(kColThreads)
    k_col_reduce_inv(const float2* __restrict__ partial, float2* __restrict__ out, int H, int Wh, int nch, int groups,
                     int TC, FftPlan pH, const float2* __restrict__ twH) {
  extern __shared__ float2 sm[];
  const int E = H * TC;
  float2* A = sm;
  float2* B = sm + E;
  const int col0 = blockIdx.x * TC, ch = blockIdx.y;
  const size_t plane = static_cast<size_t>(H) * Wh;
  for (int e = threadIdx.x; e < E; e += kColThreads) {
    const int r = e / TC, col = col0 + (e - r * TC);
    float2 s = make_float2(0.f, 0.f);
    if (col < Wh) {
      const size_t off = static_cast<size_t>(r) * Wh + col;
      for (int g = 0; g < groups; ++g) s = c_add(s, partial[(static_cast<size_t>(g) * nch + ch) * plane + off]);
    }
    A[e] = s;
  }
  __syncthreads();
  const float2* Y = stockham<+1, true>(A, B, pH, TC, TC, 1, twH, 1);
  float2* dst = out + static_cast<size_t>(ch) * plane;
  for (int e = threadIdx.x; e < E; e += kColThreads) {
    const int r = e / TC, col = col0 + (e - r * TC);
    if (col < Wh) dst[static_cast<size_t>(r) * Wh + col] = Y[e];
  }
}

// ---------------------------------------------------------------------------
// Row kernels: one CTA owns RB consecutive rows of one plane.  A real row of
// length W = 2L is handled as the complex row z[n] = x[2n] + i x[2n+1].
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(kRowThreads)
    k_row_r2c(const float* __restrict__ in, float2* __restrict__ out, int H, int L, int RB, FftPlan pL,
              const float2* __restrict__ twW, float scale) {
  extern __shared__ float2 sm[];
  const int E = RB * L, Wh = L + 1;
  float2* A = sm;
  float2* B = sm + E;
  const int row0 = blockIdx.x * RB;
  const size_t plane = blockIdx.y;
  const float2* src = reinterpret_cast<const float2*>(in) + plane * H * L;
  for (int e = threadIdx.x; e < E; e += kRowThreads) {
    const int r = e / L, row = row0 + r;
    A[e] = row < H ? src[static_cast<size_t>(row) * L + (e - r * L)] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const float2* Z = stockham<-1, false>(A, B, pL, RB, 1, L, twW, 2);
  float2* dst = out + plane * H * Wh;
  for (int e = threadIdx.x; e < RB * Wh; e += kRowThreads) {
    const int r = e / Wh, k = e - r * Wh, row = row0 + r;
    if (row < H) dst[static_cast<size_t>(row) * Wh + k] = c_scale(r2c_unpack(Z + r * L, L, k, twW), scale);
  }
}

// Loads RB packed rows of a half-spectrum plane for the inverse row transform.
__device__ __forceinline__ void load_c2r(const float2* __restrict__ src, float2* A, int H, int L, int row0, int RB,
                                         const float2* __restrict__ twW) {
  const int E = RB * L, Wh = L + 1;
  for (int e = threadIdx.x; e < E; e += kRowThreads) {
    const int r = e / L, row = row0 + r;
    A[e] = row < H ? c2r_pack(src + static_cast<size_t>(row) * Wh, L, e - r * L, twW) : make_float2(0.f, 0.f);
  }
}

__global__ void __launch_bounds__(kRowThreads)
    k_row_c2r(const float2* __restrict__ in, float* __restrict__ out, int H, int L, int RB, FftPlan pL,
              const float2* __restrict__ twW, float scale) {
  extern __shared__ float2 sm[];
  const int E = RB * L, Wh = L + 1;
  float2* A = sm;
  float2* B = sm + E;
  const int row0 = blockIdx.x * RB;
  const size_t plane = blockIdx.y;
  load_c2r(in + plane * H * Wh, A, H, L, row0, RB, twW);
  __syncthreads();
  const float2* Z = stockham<+1, false>(A, B, pL, RB, 1, L, twW, 2);
  float2* dst = reinterpret_cast<float2*>(out) + plane * H * L;
  for (int e = threadIdx.x; e < E; e += kRowThreads) {
    const int r = e / L, row = row0 + r;
    if (row < H) dst[static_cast<size_t>(row) * L + (e - r * L)] = c_scale(Z[e], scale);
  }
}

// v-step and b_v update (Sec. 3): with c = (S u)_f on this row,
// g = b_v + c, b_v <- clip(g, -t, t) = g - soft(g, t), d = soft(g) - clip(g);
// d (= v - b_v of the new iterate) is transformed back in place.
__global__ void __launch_bounds__(kRowThreads)
    k_row_shrink(float2* __restrict__ Y, float* __restrict__ bv, const float* __restrict__ thr, int eta, int H, int L,
                 int RB, FftPlan pL, const float2* __restrict__ twW, float scale, float* __restrict__ gout) {
  extern __shared__ float2 sm[];
  const int E = RB * L, Wh = L + 1;
  float2* A = sm;
  float2* B = sm + E;
  const int row0 = blockIdx.x * RB;
  const size_t plane = blockIdx.y;
  float2* X = Y + plane * H * Wh;
  load_c2r(X, A, H, L, row0, RB, twW);
  __syncthreads();
  float2* Z = stockham<+1, false>(A, B, pL, RB, 1, L, twW, 2);
  const float t = thr[plane % eta];
  float2* b2 = reinterpret_cast<float2*>(bv) + plane * H * L;
  for (int e = threadIdx.x; e < E; e += kRowThreads) {
    const int r = e / L, row = row0 + r;
    float2 d = make_float2(0.f, 0.f);
    if (row < H) {
      const size_t off = static_cast<size_t>(row) * L + (e - r * L);
      const float2 b = b2[off];
      const float gx = b.x + scale * Z[e].x, gy = b.y + scale * Z[e].y;
      const float cx = fminf(fmaxf(gx, -t), t), cy = fminf(fmaxf(gy, -t), t);
      b2[off] = make_float2(cx, cy);
      if (gout) reinterpret_cast<float2*>(gout)[plane * H * L + off] = make_float2(gx, gy);
      d = make_float2(gx - 2.f * cx, gy - 2.f * cy);
    }
    Z[e] = d;
  }
  __syncthreads();
  float2* other = (Z == A) ? B : A;
  const float2* D = stockham<-1, false>(Z, other, pL, RB, 1, L, twW, 2);
  for (int e = threadIdx.x; e < RB * Wh; e += kRowThreads) {
    const int r = e / Wh, k = e - r * Wh, row = row0 + r;
    if (row < H) X[static_cast<size_t>(row) * Wh + k] = r2c_unpack(D + r * L, L, k, twW);
  }
}

constexpr int kL1Threads = kRowThreads;

// Weighted l1 norm of the real planes behind the half spectra: one FP64
// partial per block, fixed summation order.
__global__ void __launch_bounds__(kRowThreads)
    k_row_l1(const float2* __restrict__ in, const float* __restrict__ lam, int eta, int H, int L, int RB, FftPlan pL,
             const float2* __restrict__ twW, float scale, double* __restrict__ partial) {
  extern __shared__ float2 sm[];
  __shared__ double red[kL1Threads];
  const int E = RB * L, Wh = L + 1;
  float2* A = sm;
  float2* B = sm + E;
  const int row0 = blockIdx.x * RB;
  const size_t plane = blockIdx.y;
  load_c2r(in + plane * H * Wh, A, H, L, row0, RB, twW);
  __syncthreads();
  const float2* Z = stockham<+1, false>(A, B, pL, RB, 1, L, twW, 2);
  double acc = 0.0;
  for (int e = threadIdx.x; e < E; e += kRowThreads) {
    const int r = e / L, row = row0 + r;
    if (row < H) acc += static_cast<double>(fabsf(scale * Z[e].x)) + static_cast<double>(fabsf(scale * Z[e].y));
  }
  red[threadIdx.x] = acc * static_cast<double>(lam[plane % eta]);
  __syncthreads();
  for (int s = kL1Threads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[plane * gridDim.x + blockIdx.x] = red[0];
}

// u-step (u = 1/2 [S^T(v - b_v) + (w - b_w) - gamma s], A^T A = 2I), w-step
// (pixelwise projection of g_w = b_w + u onto the simplex), b_w = g_w - w,
// and the row-forward transform of u for the next analysis.  Shared memory:
// A, B (RB x L complex each) and U (K x RB x L complex).
__global__ void __launch_bounds__(kRowThreads)
    k_row_ustep(const float2* __restrict__ T, const float* __restrict__ s, float* __restrict__ w,
                float* __restrict__ bw, float* __restrict__ u, float2* __restrict__ Ur, float* __restrict__ stv, int K,
                int H, int L, int RB, FftPlan pL, const float2* __restrict__ twW, float scale, float gamma) {
  extern __shared__ float2 sm[];
  const int E = RB * L, Wh = L + 1;
  float2* A = sm;
  float2* B = sm + E;
  float2* U = sm + 2 * E;
  const int row0 = blockIdx.x * RB;
  const size_t HL = static_cast<size_t>(H) * L, HWh = static_cast<size_t>(H) * Wh;
  for (int k = 0; k < K; ++k) {
    load_c2r(T + k * HWh, A, H, L, row0, RB, twW);
    __syncthreads();
    const float2* Z = stockham<+1, false>(A, B, pL, RB, 1, L, twW, 2);
    for (int e = threadIdx.x; e < E; e += kRowThreads) U[k * E + e] = c_scale(Z[e], scale);
    __syncthreads();
  }
  const float2* s2 = reinterpret_cast<const float2*>(s);
  float2* w2 = reinterpret_cast<float2*>(w);
  float2* bw2 = reinterpret_cast<float2*>(bw);
  float2* u2 = reinterpret_cast<float2*>(u);
  float2* stv2 = reinterpret_cast<float2*>(stv);
  const float hg = 0.5f * gamma;
  for (int e = threadIdx.x; e < E; e += kRowThreads) {
    const int r = e / L, row = row0 + r;
    if (row >= H) {
      for (int k = 0; k < K; ++k) U[k * E + e] = make_float2(0.f, 0.f);
      continue;
    }
    const size_t off = static_cast<size_t>(row) * L + (e - r * L);
    float gx[kMaxK], gy[kMaxK];
#pragma unroll
    for (int k = 0; k < kMaxK; ++k) {
      gx[k] = 0.f;
      gy[k] = 0.f;
      if (k < K) {
        const float2 st = U[k * E + e];
        const float2 wv = w2[k * HL + off], bv = bw2[k * HL + off], sv = s2[k * HL + off];
        const float ux = 0.5f * (st.x + (wv.x - bv.x)) - hg * sv.x;
        const float uy = 0.5f * (st.y + (wv.y - bv.y)) - hg * sv.y;
        u2[k * HL + off] = make_float2(ux, uy);
        if (stv) stv2[k * HL + off] = st;
        U[k * E + e] = make_float2(ux, uy);
        gx[k] = bv.x + ux;
        gy[k] = bv.y + uy;
      }
    }
    float px[kMaxK], py[kMaxK];
#pragma unroll
    for (int k = 0; k < kMaxK; ++k) {
      px[k] = gx[k];
      py[k] = gy[k];
    }
    simplex_project<kMaxK>(px, K);
    simplex_project<kMaxK>(py, K);
#pragma unroll
    for (int k = 0; k < kMaxK; ++k) {
      if (k < K) {
        w2[k * HL + off] = make_float2(px[k], py[k]);
        bw2[k * HL + off] = make_float2(gx[k] - px[k], gy[k] - py[k]);
      }
    }
  }
  __syncthreads();
  for (int k = 0; k < K; ++k) {
    const float2* Z = stockham<-1, false>(U + k * E, A, pL, RB, 1, L, twW, 2);
    float2* dst = Ur + k * HWh;
    for (int e = threadIdx.x; e < RB * Wh; e += kRowThreads) {
      const int r = e / Wh, kk = e - r * Wh, row = row0 + r;
      if (row < H) dst[static_cast<size_t>(row) * Wh + kk] = r2c_unpack(Z + r * L, L, kk, twW);
    }
    __syncthreads();
  }
}

template <typename K>
cudaError_t set_smem(K kernel, int bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

int ustep_rows(const Geo& g, int K) {
  int rb = 65536 / (g.L * (8 * K + 16));
  if (rb < 1) rb = 1;
  if (rb > g.RB) rb = g.RB;
  return rb;
}

}  // namespace

// Raises the dynamic shared-memory limit of every kernel to the device's
// opt-in maximum (an upper bound only), once per device, outside any capture.
cudaError_t prepare_kernels() {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  const cudaError_t errs[] = {
      set_smem(k_row_r2c, optin),          set_smem(k_row_c2r, optin),        set_smem(k_row_shrink, optin),
      set_smem(k_row_l1, optin - static_cast<int>(sizeof(double)) * kL1Threads),
      set_smem(k_col_fan<8>, optin),       set_smem(k_col_fan<16>, optin),    set_smem(k_col_fan<32>, optin),
      set_smem(k_col_gather<8>, optin),    set_smem(k_col_gather<16>, optin), set_smem(k_col_gather<32>, optin),
      set_smem(k_col_reduce_inv, optin),   set_smem(k_row_ustep, optin)};
  for (cudaError_t x : errs)
    if (x != cudaSuccess) return x;
  return cudaSuccess;
}

int max_dynamic_smem_needed(const Geo& g, int K) {
  const int col = static_cast<int>(2 * sizeof(float2) * g.H * g.TC);
  const int row = static_cast<int>(2 * sizeof(float2) * g.RB * g.L);
  const int us = static_cast<int>(sizeof(float2) * static_cast<size_t>(ustep_rows(g, K)) * g.L * (2 + K));
  return std::max(col, std::max(row, us));
}

bool set_generic_tiles(Geo* g, int TC, int RB, int K, int smem_limit) {
  if (TC < 1 || RB < 1 || TC > g->Wh || RB > g->H) return false;
  const int per = (g->H * TC + kColThreads - 1) / kColThreads;
  if (per > 32) return false;
  Geo t = *g;
  t.TC = TC;
  t.ntiles = (t.Wh + TC - 1) / TC;
  t.maxe = per <= 8 ? 8 : (per <= 16 ? 16 : 32);
  t.RB = RB;
  const size_t col = 2 * sizeof(float2) * static_cast<size_t>(t.H) * t.TC;
  const size_t row = 2 * sizeof(float2) * static_cast<size_t>(t.RB) * t.L;
  const size_t us = sizeof(float2) * static_cast<size_t>(ustep_rows(t, K)) * t.L * (2 + K);
  const size_t lim = static_cast<size_t>(smem_limit);
  if (col > lim || row + sizeof(double) * kL1Threads > lim || us > lim) return false;
  *g = t;
  return true;
}

int default_groups(const Geo& g, int nch) {
  const int base = g.ntiles * nch;
  int G = (4 * 152 + base - 1) / base;
  if (G < 1) G = 1;
  if (G > g.eta) G = g.eta;
  const int fg = (g.eta + G - 1) / G;
  return (g.eta + fg - 1) / fg;
}

cudaError_t run_row_r2c(const Geo& g, const float* in, float2* out, int planes, float scale, cudaStream_t st) {
  const size_t smem = 2 * sizeof(float2) * g.RB * g.L;
  dim3 grid((g.H + g.RB - 1) / g.RB, planes);
  k_row_r2c<<<grid, kRowThreads, smem, st>>>(in, out, g.H, g.L, g.RB, g.planL, g.twW, scale);
  return cudaGetLastError();
}

cudaError_t run_row_c2r(const Geo& g, const float2* in, float* out, int planes, float scale, cudaStream_t st) {
  const size_t smem = 2 * sizeof(float2) * g.RB * g.L;
  dim3 grid((g.H + g.RB - 1) / g.RB, planes);
  k_row_c2r<<<grid, kRowThreads, smem, st>>>(in, out, g.H, g.L, g.RB, g.planL, g.twW, scale);
  return cudaGetLastError();
}

cudaError_t run_row_shrink(const Geo& g, float2* Y, float* bv, const float* thr, int planes, float scale,
                           cudaStream_t st, float* gout) {
  const size_t smem = 2 * sizeof(float2) * g.RB * g.L;
  dim3 grid((g.H + g.RB - 1) / g.RB, planes);
  k_row_shrink<<<grid, kRowThreads, smem, st>>>(Y, bv, thr, g.eta, g.H, g.L, g.RB, g.planL, g.twW, scale, gout);
  return cudaGetLastError();
}

cudaError_t run_row_l1(const Geo& g, const float2* Y, const float* lam, int planes, float scale, double* partial,
                       int* nblocks, cudaStream_t st) {
  const size_t smem = 2 * sizeof(float2) * g.RB * g.L;
  dim3 grid((g.H + g.RB - 1) / g.RB, planes);
  k_row_l1<<<grid, kRowThreads, smem, st>>>(Y, lam, g.eta, g.H, g.L, g.RB, g.planL, g.twW, scale, partial);
  *nblocks = grid.x * grid.y;
  return cudaGetLastError();
}

template <int MAXE>
static cudaError_t fan_t(const Geo& g, const float2* in, float2* out, int nch, int groups, cudaStream_t st) {
  const size_t smem = 2 * sizeof(float2) * g.H * g.TC;
  const int fg = (g.eta + groups - 1) / groups;
  dim3 grid(g.ntiles, nch, (g.eta + fg - 1) / fg);
  k_col_fan<MAXE><<<grid, kColThreads, smem, st>>>(in, g.bank, out, g.H, g.Wh, g.eta, g.TC, fg, g.planH, g.twH);
  return cudaGetLastError();
}

cudaError_t run_col_fan(const Geo& g, const float2* in, float2* out, int nch, int groups, cudaStream_t st) {
  if (g.maxe == 8) return fan_t<8>(g, in, out, nch, groups, st);
  if (g.maxe == 16) return fan_t<16>(g, in, out, nch, groups, st);
  return fan_t<32>(g, in, out, nch, groups, st);
}

template <int MAXE>
static cudaError_t gather_t(const Geo& g, const float2* in, float2* partial, int nch, int groups, cudaStream_t st) {
  const size_t smem = 2 * sizeof(float2) * g.H * g.TC;
  const int fg = (g.eta + groups - 1) / groups;
  dim3 grid(g.ntiles, nch, (g.eta + fg - 1) / fg);
  k_col_gather<MAXE><<<grid, kColThreads, smem, st>>>(in, g.bank, partial, g.H, g.Wh, g.eta, nch, g.TC, fg,
                                                      g.planH, g.twH);
  return cudaGetLastError();
}

cudaError_t run_col_gather(const Geo& g, const float2* in, float2* partial, int nch, int groups, cudaStream_t st) {
  if (g.maxe == 8) return gather_t<8>(g, in, partial, nch, groups, st);
  if (g.maxe == 16) return gather_t<16>(g, in, partial, nch, groups, st);
  return gather_t<32>(g, in, partial, nch, groups, st);
}

cudaError_t run_col_reduce_inv(const Geo& g, const float2* partial, float2* out, int nch, int groups,
                               cudaStream_t st) {
  const size_t smem = 2 * sizeof(float2) * g.H * g.TC;
  dim3 grid(g.ntiles, nch);
  k_col_reduce_inv<<<grid, kColThreads, smem, st>>>(partial, out, g.H, g.Wh, nch, groups, g.TC, g.planH, g.twH);
  return cudaGetLastError();
}

cudaError_t run_row_ustep(const Geo& g, const float2* T, const float* s, float* w, float* bw, float* u, float2* Ur,
                          float* stv, int K, float gamma, float scale, cudaStream_t st) {
  const int rb = ustep_rows(g, K);
  const size_t smem = sizeof(float2) * static_cast<size_t>(rb) * g.L * (2 + K);
  dim3 grid((g.H + rb - 1) / rb);
  k_row_ustep<<<grid, kRowThreads, smem, st>>>(T, s, w, bw, u, Ur, stv, K, g.H, g.L, rb, g.planL, g.twW, scale,
                                               gamma);
  return cudaGetLastError();
}

}  // namespace shf

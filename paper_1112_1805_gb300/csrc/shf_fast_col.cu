// Column transforms of the fast path: the analysis fan-out and the synthesis
// gather over the filters of a wave, and the forward/inverse column passes of
// u and of the synthesis sum (Sec. 2, eq. for S and S^T; Sec. 3, ADMM steps).
// 8-value register FFTs (shf_fft_reg.cuh) for every height; the fan and the
// gather at heights 512, 1024 and 2048 on 16-value radix-16 FFTs (shf_fft16.cuh).
#include "shf_fast.h"
#include "shf_fft16.cuh"
#include "shf_fftv.cuh"

namespace shf {
namespace fast {
namespace {

// Columns per CTA batch (8, or 4 for heights above 1024) and the CTA's
// threads: 8 values per thread, H/8 threads per column.
template <int H>
struct ColGeo {
  static constexpr int KB = reg::col_batch(H);
  static constexpr int NT = H / 8 * KB;
};
using reg::sidx;

// Per-pass twiddle table of a length-N transform, built by the whole CTA.
template <int N, int TWSTEP>
__device__ __forceinline__ void load_pass_table(float2* pt, const float2* __restrict__ tw) {
  reg::build_pass_twiddles<N, TWSTEP>(pt, tw, threadIdx.x, blockDim.x);
}

// ---------------------------------------------------------------------------
// Column kernels: a CTA of H KB/8 threads owns KB consecutive half-spectrum
// columns, KB = 8 (4 for H > 1024; thread (b, tt) holds rows tt + k H/8 of
// column KB*tile + b).  The
// internal spectra (uhat, Y, partial) use the row pitch Whp = Wh rounded up to
// 8, so that each row segment of a tile is one aligned 64-byte piece; Ur and T,
// shared with the generic kernels, use the pitch Wh.  Global operands of the
// next filter are loaded while the current transform runs.
// ---------------------------------------------------------------------------

// Resident CTAs of NT threads (whole warps) to ask for: 32 warps per SM (64
// registers per thread) for powers of two; for H = 3 2^a or 5 2^a, whose
// radix-R pass holds more values, about 80 registers per thread.
constexpr int col_min_blocks(int H, int NT) {
  return reg::odd_part(H) == 1
             ? (32 / ((NT + 31) / 32) > 32 ? 32 : (32 / ((NT + 31) / 32) > 0 ? 32 / ((NT + 31) / 32) : 1))
             : ((65536 / 80) / (32 * ((NT + 31) / 32)) > 0 ? (65536 / 80) / (32 * ((NT + 31) / 32)) : 1);
}

template <int H>
__global__ void __launch_bounds__(ColGeo<H>::NT) k_fcol_fwd(const float2* __restrict__ in, float2* __restrict__ out, int Wh,
                                                int Whp, const float2* __restrict__ twH) {
  extern __shared__ float2 sm[];
  float2* tw = sm;  // per-pass twiddles
  float2* b0 = sm + reg::Passes<H>::TWSIZE;
  float2* b1 = b0 + reg::batch_rows(H) * ColGeo<H>::KB;
  constexpr int KB = ColGeo<H>::KB;
  const int b = threadIdx.x % KB, tt = threadIdx.x / KB;
  const int col = blockIdx.x * KB + b;
  const bool ok = col < Wh;
  const float2* src = in + static_cast<size_t>(H) * Wh * blockIdx.y + col;
  load_pass_table<H, 1>(tw, twH);
  pdl_wait();
  pdl_trigger();
  float2 v[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = ok ? src[static_cast<size_t>(tt + k * (H / 8)) * Wh] : make_float2(0.f, 0.f);
  __syncthreads();
  reg::fft<H, -1, KB>(v, tt, b, b0, b1, tw);
  if (ok) {
    float2* dst = out + static_cast<size_t>(H) * Whp * blockIdx.y + col;
#pragma unroll
    for (int k = 0; k < 8; ++k) dst[static_cast<size_t>(tt + k * (H / 8)) * Whp] = v[k];
  }
}

template <int H>
__device__ __forceinline__ void load_bank8(float (&w)[8], const float* __restrict__ wf, int Wh, int tt, int col,
                                           bool ok) {
#pragma unroll
  for (int k = 0; k < 8; ++k) w[k] = ok ? __ldg(wf + static_cast<size_t>(tt + k * (H / 8)) * Wh + col) : 0.f;
}

template <int H>
__device__ __forceinline__ void load_tile8(float2 (&v)[8], const float2* __restrict__ src, int pitch, int tt,
                                           int col, bool ok) {
#pragma unroll
  for (int k = 0; k < 8; ++k)
    v[k] = ok ? src[static_cast<size_t>(tt + k * (H / 8)) * pitch + col] : make_float2(0.f, 0.f);
}

// Analysis fan-out: for every item (label, tile, filter) of the CTA's range,
// Y_v = column-inverse(W_f * uhat_label) on the tile, v = (label - l0) nf +
// (f - f0).  The next item's filter tile (and, at a change of tile or label,
// the next spectrum tile) is requested while the current transform runs.
template <int H>
__global__ void __launch_bounds__(ColGeo<H>::NT, col_min_blocks(H, ColGeo<H>::NT))
    k_fcol_fan(const float2* __restrict__ uhat, const float* __restrict__ bank, const WorkItem* __restrict__ items,
               const int* __restrict__ cta_begin, float2* __restrict__ Y, int Wh, int Whp, int l0, int f0, int nf,
               const float2* __restrict__ twH) {
  extern __shared__ float2 sm[];
  float2* tw = sm;  // per-pass twiddles
  float2* b0 = sm + reg::Passes<H>::TWSIZE;
  float2* b1 = b0 + reg::batch_rows(H) * ColGeo<H>::KB;
  const int ib = cta_begin[blockIdx.x], ie = cta_begin[blockIdx.x + 1];
  if (ib >= ie) return;
  constexpr int KB = ColGeo<H>::KB;
  const int b = threadIdx.x % KB, tt = threadIdx.x / KB;
  const size_t Pb = static_cast<size_t>(H) * Wh, Pp = static_cast<size_t>(H) * Whp;
  WorkItem it = items[ib];
  int col = it.tile * KB + b;
  bool ok = col < Wh;
  float2 u[8];
  float w[8];
  load_bank8<H>(w, bank + Pb * it.filter, Wh, tt, col, ok);
  load_pass_table<H, 1>(tw, twH);
  pdl_wait();
  pdl_trigger();
  load_tile8<H>(u, uhat + Pp * it.label, Whp, tt, col, ok);
  __syncthreads();
  for (int i = ib; i < ie; ++i) {
    float2 v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = c_scale(u[k], w[k]);
    const int fl = (it.label - l0) * nf + (it.filter - f0), ccol = col;
    const bool cok = ok;
    if (i + 1 < ie) {
      const WorkItem nx = items[i + 1];
      col = nx.tile * KB + b;
      ok = col < Wh;
      load_bank8<H>(w, bank + Pb * nx.filter, Wh, tt, col, ok);
      if (nx.tile != it.tile || nx.label != it.label) load_tile8<H>(u, uhat + Pp * nx.label, Whp, tt, col, ok);
      it = nx;
    }
    reg::fft<H, +1, KB>(v, tt, b, b0, b1, tw);
    if (cok) {
      float2* dst = Y + Pp * fl + ccol;
#pragma unroll
      for (int k = 0; k < 8; ++k) dst[static_cast<size_t>(tt + k * (H / 8)) * Whp] = v[k];
    }
  }
}

// The analysis fan-out with 16 values per thread (heights 512, 1024 and 2048:
// radix-16 column transforms, one exchange fewer at 1024 and 2048): CTAs of
// KB H/16 threads (KB = 8, or 4 at 2048), thread (b, tt) holding rows
// tt + k H/16 of column b.  Measured at
// 512 x 512: 3667 -> 3721 Mpixel*label*iter/s; at 256 (unrolled 256 x 256
// sweeps) neutral, so 256 keeps the 8-value kernel.
template <int H>
struct Col16Geo {
  static constexpr int KB = reg::col_batch(H);  // the plan's column tile: 8, or 4 above 1024
  static constexpr int T = H / 16;
  static constexpr int NT = KB * T;
  static constexpr int PT = (r16::Passes<H>::TWSIZE + 1) & ~1;  // per-pass twiddles
  static constexpr int BR = r16::brows16(H) * KB;                // one exchange buffer
  static constexpr int TOTAL = PT + 2 * BR;
};
__host__ __device__ constexpr bool use_fan16(int H) { return H == 512 || H == 1024 || H == 2048; }
__host__ __device__ constexpr int fan16_len(int H) { return use_fan16(H) ? H : 512; }

template <int H>
__global__ void __launch_bounds__(Col16Geo<H>::NT, H == 512 ? 2 : 1)
    k_fcol_fan16(const float2* __restrict__ uhat, const float* __restrict__ bank, const WorkItem* __restrict__ items,
                 const int* __restrict__ cta_begin, float2* __restrict__ Y, int Wh, int Whp, int l0, int f0, int nf,
                 const float2* __restrict__ twH) {
  using G = Col16Geo<H>;
  constexpr int KB = G::KB, T = G::T;
  extern __shared__ __align__(16) float2 sm[];
  float2* pt = sm;
  float2* b0 = sm + G::PT;
  float2* b1 = b0 + G::BR;
  const int ib = cta_begin[blockIdx.x], ie = cta_begin[blockIdx.x + 1];
  if (ib >= ie) return;
  const int b = threadIdx.x % KB, tt = threadIdx.x / KB;
  const size_t Pb = static_cast<size_t>(H) * Wh, Pp = static_cast<size_t>(H) * Whp;
  WorkItem it = items[ib];
  int col = it.tile * KB + b;
  bool ok = col < Wh;
  float2 u[16];
  float w[16];
  auto load_w = [&](const float* wf, int c, bool o) {
#pragma unroll
    for (int k = 0; k < 16; ++k) w[k] = o ? __ldg(wf + static_cast<size_t>(tt + k * T) * Wh + c) : 0.f;
  };
  auto load_u = [&](const float2* src, int c, bool o) {
#pragma unroll
    for (int k = 0; k < 16; ++k) u[k] = o ? src[static_cast<size_t>(tt + k * T) * Whp + c] : make_float2(0.f, 0.f);
  };
  load_w(bank + Pb * it.filter, col, ok);
  r16::build_pass_twiddles<H, 1>(pt, twH, threadIdx.x, blockDim.x);
  pdl_wait();
  pdl_trigger();
  load_u(uhat + Pp * it.label, col, ok);
  for (int i = ib; i < ie; ++i) {
    float2 v[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = c_scale(u[k], w[k]);
    const int fl = (it.label - l0) * nf + (it.filter - f0), ccol = col;
    const bool cok = ok;
    if (i + 1 < ie) {
      const WorkItem nx = items[i + 1];
      col = nx.tile * KB + b;
      ok = col < Wh;
      load_w(bank + Pb * nx.filter, col, ok);
      if (nx.tile != it.tile || nx.label != it.label) load_u(uhat + Pp * nx.label, col, ok);
      it = nx;
    }
    r16::batch_fft<H, +1, KB>(v, tt, b, b0, b1, pt);  // starts with a CTA barrier (also after the twiddle table)
    if (cok) {
      float2* dst = Y + Pp * fl + ccol;
      const uint64_t keep = l2_evict_last_policy();
#pragma unroll
      for (int k = 0; k < 16; ++k) st_l2_hint(dst + static_cast<size_t>(tt + k * T) * Whp, v[k], keep);
    }
  }
}

// Synthesis gather: partial[slot] = sum over a run of items of one (label,
// tile) of W_f * column-forward(Y_v), stored compactly as [H][KB]; the next
// item's coefficient tile is requested while the current transform runs.
// The gather keeps its run accumulator, the prefetched tile and the transform
// in registers: it asks for half the fan's CTAs per SM, i.e. twice the
// registers (at 512 x 512: 69 against 78 us per iteration).
constexpr int gather_min_blocks(int H, int NT) { return col_min_blocks(H, NT) > 1 ? col_min_blocks(H, NT) / 2 : 1; }

template <int H>
__global__ void __launch_bounds__(ColGeo<H>::NT, gather_min_blocks(H, ColGeo<H>::NT))
    k_fcol_gather(const float2* __restrict__ Y, const float* __restrict__ bank, const WorkItem* __restrict__ items,
                  const int* __restrict__ cta_begin, float2* __restrict__ partial, int Wh, int Whp, int l0, int f0,
                  int nf, const float2* __restrict__ twH) {
  extern __shared__ float2 sm[];
  float2* tw = sm;  // per-pass twiddles
  float2* b0 = sm + reg::Passes<H>::TWSIZE;
  float2* b1 = b0 + reg::batch_rows(H) * ColGeo<H>::KB;
  const int ib = cta_begin[blockIdx.x], ie = cta_begin[blockIdx.x + 1];
  if (ib >= ie) return;
  constexpr int KB = ColGeo<H>::KB;
  const int b = threadIdx.x % KB, tt = threadIdx.x / KB;
  const size_t Pb = static_cast<size_t>(H) * Wh, Pp = static_cast<size_t>(H) * Whp;
  WorkItem it = items[ib];
  int col = it.tile * KB + b;
  bool ok = col < Wh;
  float2 acc[8], y[8];
  float w[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) acc[k] = make_float2(0.f, 0.f);
  load_pass_table<H, 1>(tw, twH);
  pdl_wait();
  pdl_trigger();
  load_tile8<H>(y, Y + Pp * ((it.label - l0) * nf + (it.filter - f0)), Whp, tt, col, ok);
  __syncthreads();
  for (int i = ib; i < ie; ++i) {
    float2 v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = y[k];
    load_bank8<H>(w, bank + Pb * it.filter, Wh, tt, col, ok);
    WorkItem nx = it;
    int ncol = col;
    bool nok = ok;
    if (i + 1 < ie) {
      nx = items[i + 1];
      ncol = nx.tile * KB + b;
      nok = ncol < Wh;
      load_tile8<H>(y, Y + Pp * ((nx.label - l0) * nf + (nx.filter - f0)), Whp, tt, ncol, nok);
    }
    reg::fft<H, -1, KB>(v, tt, b, b0, b1, tw);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      acc[k].x = fmaf(w[k], v[k].x, acc[k].x);
      acc[k].y = fmaf(w[k], v[k].y, acc[k].y);
    }
    if (i + 1 == ie || nx.slot != it.slot) {
      float2* dst = partial + static_cast<size_t>(it.slot) * H * KB + b;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        dst[static_cast<size_t>(tt + k * (H / 8)) * KB] = acc[k];
        acc[k] = make_float2(0.f, 0.f);
      }
    }
    it = nx;
    col = ncol;
    ok = nok;
  }
}

// The synthesis gather with 16 values per thread (heights 512, 1024, 2048), on
// the fan's radix-16 geometry (two CTAs of 256 threads per SM at 512, with
// 128 registers for the prefetched tile, the accumulator and the transform).
// Measured at 512 x 512: gather 69.5 -> 65.5 us per iteration, 3739 -> 3758
// Mpixel*label*iter/s (more gather CTAs leave more slots to the reduction).
template <int H>
__global__ void __launch_bounds__(Col16Geo<H>::NT, H == 512 ? 2 : 1)
    k_fcol_gather16(const float2* __restrict__ Y, const float* __restrict__ bank,
                    const WorkItem* __restrict__ items, const int* __restrict__ cta_begin,
                    float2* __restrict__ partial, int Wh, int Whp, int l0, int f0, int nf,
                    const float2* __restrict__ twH) {
  using G = Col16Geo<H>;
  constexpr int KB = G::KB, T = G::T;
  extern __shared__ __align__(16) float2 sm[];
  float2* pt = sm;
  float2* b0 = sm + G::PT;
  float2* b1 = b0 + G::BR;
  const int ib = cta_begin[blockIdx.x], ie = cta_begin[blockIdx.x + 1];
  if (ib >= ie) return;
  const int b = threadIdx.x % KB, tt = threadIdx.x / KB;
  const size_t Pb = static_cast<size_t>(H) * Wh, Pp = static_cast<size_t>(H) * Whp;
  WorkItem it = items[ib];
  int col = it.tile * KB + b;
  bool ok = col < Wh;
  float2 acc[16], y[16];
  float w[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) acc[k] = make_float2(0.f, 0.f);
  auto load_y = [&](const float2* src, int c, bool o) {
    const uint64_t last = l2_evict_first_policy();
#pragma unroll
    for (int k = 0; k < 16; ++k)
      y[k] = o ? ld_l2_hint(src + static_cast<size_t>(tt + k * T) * Whp + c, last) : make_float2(0.f, 0.f);
  };
  r16::build_pass_twiddles<H, 1>(pt, twH, threadIdx.x, blockDim.x);
  pdl_wait();
  pdl_trigger();
  load_y(Y + Pp * ((it.label - l0) * nf + (it.filter - f0)), col, ok);
  for (int i = ib; i < ie; ++i) {
    float2 v[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = y[k];
#pragma unroll
    for (int k = 0; k < 16; ++k)
      w[k] = ok ? __ldg(bank + Pb * it.filter + static_cast<size_t>(tt + k * T) * Wh + col) : 0.f;
    WorkItem nx = it;
    int ncol = col;
    bool nok = ok;
    if (i + 1 < ie) {
      nx = items[i + 1];
      ncol = nx.tile * KB + b;
      nok = ncol < Wh;
      load_y(Y + Pp * ((nx.label - l0) * nf + (nx.filter - f0)), ncol, nok);
    }
    r16::batch_fft<H, -1, KB>(v, tt, b, b0, b1, pt);  // starts with a CTA barrier (also after the twiddle table)
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      acc[k].x = fmaf(w[k], v[k].x, acc[k].x);
      acc[k].y = fmaf(w[k], v[k].y, acc[k].y);
    }
    if (i + 1 == ie || nx.slot != it.slot) {
      float2* dst = partial + static_cast<size_t>(it.slot) * H * KB + b;
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        dst[static_cast<size_t>(tt + k * T) * KB] = acc[k];
        acc[k] = make_float2(0.f, 0.f);
      }
    }
    it = nx;
    col = ncol;
    ok = nok;
  }
}

// The fan and the gather with V = 12 or 20 values per thread for the heights
// with an odd factor (H = 12 T or 20 T, T = 2..128: shf_fftv.cuh), on the
// geometry of the radix-16 kernels: CTAs of KB H/V threads, thread (b, tt)
// holding rows tt + k H/V of column b.  Resident CTAs are asked for with at
// most 128 registers per thread.
template <int H>
struct ColVGeo {
  static constexpr int KB = reg::col_batch(H);
  static constexpr int V = rv::vals_for(H);
  static constexpr int T = H / V;
  static constexpr int NT = KB * T;
  static constexpr int PT = (rv::Passes<H>::TWSIZE + 1) & ~1;  // per-pass twiddles
  static constexpr int BR = rv::brows(H) * KB;                 // one exchange buffer
  static constexpr int TOTAL = PT + 2 * BR;
  static constexpr int WARPS = (NT + 31) / 32;
  static constexpr int MINB = 16 / WARPS > 1 ? 16 / WARPS : 1;  // 128 registers per thread
};
__host__ __device__ constexpr bool use_colv(int H) { return rv::supported_col(H); }
__host__ __device__ constexpr int colv_len(int H) { return use_colv(H) ? H : 24; }

template <int H>
__global__ void __launch_bounds__(ColVGeo<H>::NT, ColVGeo<H>::MINB)
    k_fcol_fanv(const float2* __restrict__ uhat, const float* __restrict__ bank, const WorkItem* __restrict__ items,
                const int* __restrict__ cta_begin, float2* __restrict__ Y, int Wh, int Whp, int l0, int f0, int nf,
                const float2* __restrict__ twH) {
  using G = ColVGeo<H>;
  constexpr int KB = G::KB, T = G::T, V = G::V;
  extern __shared__ __align__(16) float2 sm[];
  float2* pt = sm;
  float2* b0 = sm + G::PT;
  float2* b1 = b0 + G::BR;
  const int ib = cta_begin[blockIdx.x], ie = cta_begin[blockIdx.x + 1];
  if (ib >= ie) return;
  const int b = threadIdx.x % KB, tt = threadIdx.x / KB;
  const size_t Pb = static_cast<size_t>(H) * Wh, Pp = static_cast<size_t>(H) * Whp;
  WorkItem it = items[ib];
  int col = it.tile * KB + b;
  bool ok = col < Wh;
  float2 u[V];
  float w[V];
  auto load_w = [&](const float* wf, int c, bool o) {
#pragma unroll
    for (int k = 0; k < V; ++k) w[k] = o ? __ldg(wf + static_cast<size_t>(tt + k * T) * Wh + c) : 0.f;
  };
  auto load_u = [&](const float2* src, int c, bool o) {
#pragma unroll
    for (int k = 0; k < V; ++k) u[k] = o ? src[static_cast<size_t>(tt + k * T) * Whp + c] : make_float2(0.f, 0.f);
  };
  load_w(bank + Pb * it.filter, col, ok);
  rv::build_pass_twiddles<H, 1>(pt, twH, threadIdx.x, blockDim.x);
  pdl_wait();
  pdl_trigger();
  load_u(uhat + Pp * it.label, col, ok);
  for (int i = ib; i < ie; ++i) {
    float2 v[V];
#pragma unroll
    for (int k = 0; k < V; ++k) v[k] = c_scale(u[k], w[k]);
    const int fl = (it.label - l0) * nf + (it.filter - f0), ccol = col;
    const bool cok = ok;
    if (i + 1 < ie) {
      const WorkItem nx = items[i + 1];
      col = nx.tile * KB + b;
      ok = col < Wh;
      load_w(bank + Pb * nx.filter, col, ok);
      if (nx.tile != it.tile || nx.label != it.label) load_u(uhat + Pp * nx.label, col, ok);
      it = nx;
    }
    rv::batch_fft<H, +1, KB>(v, tt, b, b0, b1, pt);  // starts with a CTA barrier (also after the twiddle table)
    if (cok) {
      float2* dst = Y + Pp * fl + ccol;
      const uint64_t keep = l2_evict_last_policy();
#pragma unroll
      for (int k = 0; k < V; ++k) st_l2_hint(dst + static_cast<size_t>(tt + k * T) * Whp, v[k], keep);
    }
  }
}

// The gather keeps the next item's tile in registers while the current one
// is transformed for V = 12; for V = 20 the run accumulator, the filter column
// and the transform already take 100 registers, and the tile is loaded when
// its item starts.
template <int H>
__global__ void __launch_bounds__(ColVGeo<H>::NT, ColVGeo<H>::MINB)
    k_fcol_gatherv(const float2* __restrict__ Y, const float* __restrict__ bank, const WorkItem* __restrict__ items,
                   const int* __restrict__ cta_begin, float2* __restrict__ partial, int Wh, int Whp, int l0, int f0,
                   int nf, const float2* __restrict__ twH) {
  using G = ColVGeo<H>;
  constexpr int KB = G::KB, T = G::T, V = G::V;
  constexpr bool PREFETCH = V <= 12;
  extern __shared__ __align__(16) float2 sm[];
  float2* pt = sm;
  float2* b0 = sm + G::PT;
  float2* b1 = b0 + G::BR;
  const int ib = cta_begin[blockIdx.x], ie = cta_begin[blockIdx.x + 1];
  if (ib >= ie) return;
  const int b = threadIdx.x % KB, tt = threadIdx.x / KB;
  const size_t Pb = static_cast<size_t>(H) * Wh, Pp = static_cast<size_t>(H) * Whp;
  WorkItem it = items[ib];
  int col = it.tile * KB + b;
  bool ok = col < Wh;
  float2 acc[V], y[PREFETCH ? V : 1];
  float w[V];
#pragma unroll
  for (int k = 0; k < V; ++k) acc[k] = make_float2(0.f, 0.f);
  auto tile_of = [&](const WorkItem& x) { return Y + Pp * ((x.label - l0) * nf + (x.filter - f0)); };
  const uint64_t last = l2_evict_first_policy();  // the spectra's last reader
  rv::build_pass_twiddles<H, 1>(pt, twH, threadIdx.x, blockDim.x);
  pdl_wait();
  pdl_trigger();
  if constexpr (PREFETCH) {
    const float2* src = tile_of(it);
#pragma unroll
    for (int k = 0; k < V; ++k) y[k] = ok ? ld_l2_hint(src + static_cast<size_t>(tt + k * T) * Whp + col, last) : make_float2(0.f, 0.f);
  }
  for (int i = ib; i < ie; ++i) {
    float2 v[V];
    if constexpr (PREFETCH) {
#pragma unroll
      for (int k = 0; k < V; ++k) v[k] = y[k];
    } else {
      const float2* src = tile_of(it);
#pragma unroll
      for (int k = 0; k < V; ++k) v[k] = ok ? ld_l2_hint(src + static_cast<size_t>(tt + k * T) * Whp + col, last) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int k = 0; k < V; ++k)
      w[k] = ok ? __ldg(bank + Pb * it.filter + static_cast<size_t>(tt + k * T) * Wh + col) : 0.f;
    WorkItem nx = it;
    int ncol = col;
    bool nok = ok;
    if (i + 1 < ie) {
      nx = items[i + 1];
      ncol = nx.tile * KB + b;
      nok = ncol < Wh;
      if constexpr (PREFETCH) {
        const float2* src = tile_of(nx);
#pragma unroll
        for (int k = 0; k < V; ++k)
          y[k] = nok ? ld_l2_hint(src + static_cast<size_t>(tt + k * T) * Whp + ncol, last) : make_float2(0.f, 0.f);
      }
    }
    rv::batch_fft<H, -1, KB>(v, tt, b, b0, b1, pt);  // starts with a CTA barrier (also after the twiddle table)
#pragma unroll
    for (int k = 0; k < V; ++k) {
      acc[k].x = fmaf(w[k], v[k].x, acc[k].x);
      acc[k].y = fmaf(w[k], v[k].y, acc[k].y);
    }
    if (i + 1 == ie || nx.slot != it.slot) {
      float2* dst = partial + static_cast<size_t>(it.slot) * H * KB + b;
#pragma unroll
      for (int k = 0; k < V; ++k) {
        dst[static_cast<size_t>(tt + k * T) * KB] = acc[k];
        acc[k] = make_float2(0.f, 0.f);
      }
    }
    it = nx;
    col = ncol;
    ok = nok;
  }
}

// T[label] on one tile = column-inverse of the sum of the tile's partial
// slots, in a fixed order.  The sum is load-latency bound (and small images
// have few tiles), so the slots are split into RG consecutive runs (RG copies
// of the CTA's threads, up to 4, within 1024 threads) summed by RG thread
// groups at once; the first group adds the other groups' sums in group order
// and transforms.  The other groups run the same transform on their own
// buffers (their results are discarded), so that all pass the same barriers.
template <int H>
struct ReduceGeo {
  static constexpr int NT = ColGeo<H>::NT;
  static constexpr int RG = 1024 / NT >= 4 ? 4 : (1024 / NT >= 1 ? 1024 / NT : 1);
  static constexpr int BR = reg::batch_rows(H) * ColGeo<H>::KB;       // one exchange buffer
  static constexpr int BUFS = (reg::Passes<H>::TWSIZE + 1) & ~1;     // offset of the buffers
  static constexpr int STAGE = BUFS + 2 * RG * BR;                    // groups 1.. : their sums [H][KB]
  static constexpr int TOTAL = STAGE + (RG - 1) * H * ColGeo<H>::KB;
};

template <int H>
__global__ void __launch_bounds__(ReduceGeo<H>::RG * ColGeo<H>::NT) k_fcol_reduce_inv(
    const float2* __restrict__ partial, const int* __restrict__ tile_begin, const int* __restrict__ tile_slots,
    float2* __restrict__ T, int Wh, const float2* __restrict__ twH) {
  using RGeo = ReduceGeo<H>;
  constexpr int KB = ColGeo<H>::KB;
  constexpr int NT = ColGeo<H>::NT;
  extern __shared__ __align__(16) float2 sm[];
  float2* tw = sm;  // per-pass twiddles
  const int grp = threadIdx.x / NT, lt = threadIdx.x - grp * NT;
  float2* b0 = sm + RGeo::BUFS + 2 * grp * RGeo::BR;
  float2* b1 = b0 + RGeo::BR;
  float2* stage = sm + RGeo::STAGE;
  const int b = lt % KB, tt = lt / KB;
  const int tile = blockIdx.x, label = blockIdx.y;
  const int col = tile * KB + b;
  const bool ok = col < Wh;
  float2 v[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = make_float2(0.f, 0.f);
  load_pass_table<H, 1>(tw, twH);
  pdl_wait();
  pdl_trigger();
  const int lt0 = label * gridDim.x + tile;  // the (label, tile) slot list
  const int s0 = tile_begin[lt0], s1 = tile_begin[lt0 + 1], ns = s1 - s0;
  const int a0 = s0 + ns * grp / RGeo::RG, a1 = s0 + ns * (grp + 1) / RGeo::RG;
  for (int si = a0; si < a1; ++si) {
    const float2* src = partial + static_cast<size_t>(tile_slots[si]) * H * KB + b;
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = c_add(v[k], src[static_cast<size_t>(tt + k * (H / 8)) * KB]);
  }
  if constexpr (RGeo::RG > 1) {
    if (grp > 0) {
      float2* st = stage + (grp - 1) * H * KB;
#pragma unroll
      for (int k = 0; k < 8; ++k) st[(tt + k * (H / 8)) * KB + b] = v[k];
    }
    __syncthreads();
    if (grp == 0) {
      for (int g2 = 1; g2 < RGeo::RG; ++g2) {
        const float2* st = stage + (g2 - 1) * H * KB;
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = c_add(v[k], st[(tt + k * (H / 8)) * KB + b]);
      }
    }
  }
  __syncthreads();
  reg::fft<H, +1, KB>(v, tt, b, b0, b1, tw);
  if (grp == 0 && ok) {
    float2* dst = T + static_cast<size_t>(H) * Wh * label + col;
#pragma unroll
    for (int k = 0; k < 8; ++k) dst[static_cast<size_t>(tt + k * (H / 8)) * Wh] = v[k];
  }
}

template <int N>
size_t col_smem() {
  return sizeof(float2) * (reg::Passes<N>::TWSIZE + 2 * reg::batch_rows(N) * ColGeo<N>::KB);
}

template <int N>
size_t fan16_smem() {
  return sizeof(float2) * Col16Geo<fan16_len(N)>::TOTAL;
}

template <int N>
size_t colv_smem() {
  return sizeof(float2) * ColVGeo<colv_len(N)>::TOTAL;
}

template <int H>
cudaError_t prepare_col_t() {
  const size_t s = col_smem<H>();
  cudaError_t e = allow_smem(k_fcol_fwd<H>, s);
  if (e == cudaSuccess) e = allow_smem(k_fcol_fan<H>, s);
  if constexpr (use_fan16(H)) {
    if (e == cudaSuccess) e = allow_smem(k_fcol_fan16<H>, fan16_smem<H>());
    if (e == cudaSuccess) e = allow_smem(k_fcol_gather16<H>, fan16_smem<H>());
  }
  if constexpr (use_colv(H)) {
    if (e == cudaSuccess) e = allow_smem(k_fcol_fanv<H>, colv_smem<H>());
    if (e == cudaSuccess) e = allow_smem(k_fcol_gatherv<H>, colv_smem<H>());
  }
  if (e == cudaSuccess) e = allow_smem(k_fcol_gather<H>, s);
  if (e == cudaSuccess) e = allow_smem(k_fcol_reduce_inv<H>, sizeof(float2) * ReduceGeo<H>::TOTAL);
  return e;
}

}  // namespace

cudaError_t prepare_col_kernels() {
#define SHF_PREP(N) \
  if (e == cudaSuccess) e = prepare_col_t<N>();
  cudaError_t e = cudaSuccess;
  SHF_COL_SIZES(SHF_PREP)
#undef SHF_PREP
  return e;
}

// The column transform a plan's variant selects at height H: radix-16 (16
// values per thread) where it exists and is asked for or is the default.
bool use16(int H, int variant) { return use_fan16(H) && variant != kCol8; }
// V values per thread: asked for, or the default where it exists
bool usev(int H, int variant) { return use_colv(H) && (variant == kColV || variant == kColDefault); }

bool col_kernel_ok(int H, int variant) {
  return variant == kColDefault || variant == kCol8 || (variant == kCol16 && use_fan16(H)) ||
         (variant == kColV && use_colv(H));
}

int fan_ctas_per_sm(int H, int variant) {
  int fit = 0;
  cudaError_t e = cudaErrorInvalidValue;
  switch (H) {
#define SHF_OCC(N)                                                                                          \
  case N:                                                                                                   \
    if (use16(N, variant))                                                                                  \
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, k_fcol_fan16<fan16_len(N)>,                  \
                                                        Col16Geo<fan16_len(N)>::NT, fan16_smem<N>());      \
    else if (usev(N, variant))                                                                              \
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, k_fcol_fanv<colv_len(N)>,                    \
                                                        ColVGeo<colv_len(N)>::NT, colv_smem<N>());         \
    else                                                                                                    \
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, k_fcol_fan<N>, ColGeo<N>::NT, col_smem<N>()); \
    break;
    SHF_COL_SIZES(SHF_OCC)
#undef SHF_OCC
    default: break;
  }
  return e == cudaSuccess ? fit : 0;
}

int col_ctas_per_sm(int H, int variant) {
  int fit = 0;
  cudaError_t e = cudaErrorInvalidValue;
  switch (H) {
#define SHF_OCC(N)                                                                                          \
  case N:                                                                                                   \
    if (use16(N, variant))                                                                                  \
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, k_fcol_gather16<fan16_len(N)>,               \
                                                        Col16Geo<fan16_len(N)>::NT, fan16_smem<N>());      \
    else if (usev(N, variant))                                                                              \
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, k_fcol_gatherv<colv_len(N)>,                \
                                                        ColVGeo<colv_len(N)>::NT, colv_smem<N>());         \
    else                                                                                                    \
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, k_fcol_gather<N>, ColGeo<N>::NT, col_smem<N>()); \
    break;
    SHF_COL_SIZES(SHF_OCC)
#undef SHF_OCC
    default: break;
  }
  return e == cudaSuccess ? fit : 0;
}

cudaError_t col_fwd(const Geo& g, const float2* Ur, float2* uhat, int K, int Whp, cudaStream_t st) {
  const int tw = reg::col_batch(g.H), ntiles = (g.Wh + tw - 1) / tw;
  switch (g.H) {
#define SHF_CASE(N) \
  case N:           \
    return launch_pdl(k_fcol_fwd<N>, dim3(ntiles, K), dim3(ColGeo<N>::NT), col_smem<N>(), st, Ur, uhat, g.Wh, Whp, g.twH);
    SHF_COL_SIZES(SHF_CASE)
#undef SHF_CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t col_fan(const Geo& g, int nc, const float2* uhat, const WorkItem* items, const int* cta_begin,
                    float2* Y, int Whp, const Wave& wv, int variant, cudaStream_t st) {
  switch (g.H) {
#define SHF_CASE(N)                                                                                              \
  case N:                                                                                                        \
    if (use16(N, variant))                                                                                       \
      return launch_pdl(k_fcol_fan16<fan16_len(N)>, dim3(nc), dim3(Col16Geo<fan16_len(N)>::NT), fan16_smem<N>(),  \
                        st, uhat, g.bank, items, cta_begin, Y, g.Wh, Whp, wv.l0, wv.f0, wv.nf, g.twH);           \
    if (usev(N, variant))                                                                                        \
      return launch_pdl(k_fcol_fanv<colv_len(N)>, dim3(nc), dim3(ColVGeo<colv_len(N)>::NT), colv_smem<N>(), st,  \
                        uhat, g.bank, items, cta_begin, Y, g.Wh, Whp, wv.l0, wv.f0, wv.nf, g.twH);               \
    return launch_pdl(k_fcol_fan<N>, dim3(nc), dim3(ColGeo<N>::NT), col_smem<N>(), st, uhat, g.bank, items, cta_begin, Y, \
                      g.Wh, Whp, wv.l0, wv.f0, wv.nf, g.twH);
    SHF_COL_SIZES(SHF_CASE)
#undef SHF_CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t col_gather(const Geo& g, int nc, const float2* Y, const WorkItem* items, const int* cta_begin,
                       float2* partial, int Whp, const Wave& wv, int variant, cudaStream_t st) {
  switch (g.H) {
#define SHF_CASE(N)                                                                                           \
  case N:                                                                                                     \
    if (use16(N, variant))                                                                                    \
      return launch_pdl(k_fcol_gather16<fan16_len(N)>, dim3(nc), dim3(Col16Geo<fan16_len(N)>::NT),           \
                        fan16_smem<N>(), st, Y, g.bank, items, cta_begin, partial, g.Wh, Whp, wv.l0, wv.f0,   \
                        wv.nf, g.twH);                                                                        \
    if (usev(N, variant))                                                                                     \
      return launch_pdl(k_fcol_gatherv<colv_len(N)>, dim3(nc), dim3(ColVGeo<colv_len(N)>::NT), colv_smem<N>(), \
                        st, Y, g.bank, items, cta_begin, partial, g.Wh, Whp, wv.l0, wv.f0, wv.nf, g.twH);      \
    return launch_pdl(k_fcol_gather<N>, dim3(nc), dim3(ColGeo<N>::NT), col_smem<N>(), st, Y, g.bank, items, cta_begin, \
                      partial, g.Wh, Whp, wv.l0, wv.f0, wv.nf, g.twH);
    SHF_COL_SIZES(SHF_CASE)
#undef SHF_CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t col_reduce(const Geo& g, const float2* partial, const int* tile_begin, const int* tile_slots, float2* T,
                       int K, cudaStream_t st) {
  const int tw = reg::col_batch(g.H), ntiles = (g.Wh + tw - 1) / tw;
  switch (g.H) {
#define SHF_CASE(N)                                                                                          \
  case N:                                                                                                    \
    return launch_pdl(k_fcol_reduce_inv<N>, dim3(ntiles, K), dim3(ReduceGeo<N>::RG * ColGeo<N>::NT),             \
                      sizeof(float2) * ReduceGeo<N>::TOTAL, st, partial, tile_begin,                                  \
                      tile_slots, T, g.Wh, g.twH);
    SHF_COL_SIZES(SHF_CASE)
#undef SHF_CASE
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fast
}  // namespace shf

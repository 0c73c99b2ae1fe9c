// Fast path for power-of-two sizes (8 <= H <= 1024, 16 <= W <= 2048): the
// per-filter work of an ADMM iteration (Sec. 3 of Haeuser & Steidl) with
// register-resident FFTs (shf_fft_reg.cuh).
//
// One iteration, after the u/w-step (k_row_ustep) has left the row spectra of
// u in Ur:
//   k_fcol_fwd      Ur -> Uhat, the full 2-D spectrum of u, once per label;
//   per label k, per wave of filters [f0, f0 + nf):
//     k_fcol_fan      Y_f = column-inverse(W_f * Uhat_k) for f in the wave
//     k_wrow_shrink   row-inverse, g = b_v + S u, b_v <- clip(g), d = soft(g) -
//                     clip(g) (= v - b_v), row-forward of d, in place in Y_f
//     k_fcol_gather   partial_g += sum_{f in group g} W_f * column-forward(Y_f)
//   k_fcol_reduce_inv  T_k = column-inverse(sum_g partial_g)
// The coefficient spectra of one wave (a few tens of MB) stay in L2 between
// the three kernels; b_v is streamed with evict-first hints.
#include <algorithm>
#include <cstdint>

#include "shf_fft_reg.cuh"
#include "shf_internal.h"

namespace shf {

int fast_pitch(const Geo& g);

namespace {

using reg::kB;
using reg::kS;
using reg::sidx;

__device__ __forceinline__ void load_table(float2* dst, const float2* __restrict__ src, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

// Per-pass twiddle table of a length-N transform, built by the whole CTA.
template <int N, int TWSTEP>
__device__ __forceinline__ void load_pass_table(float2* pt, const float2* __restrict__ tw) {
  reg::build_pass_twiddles<N, TWSTEP>(pt, tw, threadIdx.x, blockDim.x);
}

// ---------------------------------------------------------------------------
// Column kernels: a CTA of H threads owns 8 consecutive half-spectrum columns
// (thread (b, tt) holds rows tt + k H/8 of column 8*blockIdx.x + b).  The
// internal spectra (uhat, Y, partial) use the row pitch Whp = Wh rounded up to
// 8, so that each row segment of a tile is one aligned 64-byte piece; Ur and T,
// shared with the generic kernels, use the pitch Wh.  Global operands of the
// next filter are loaded while the current transform runs.
// ---------------------------------------------------------------------------

// CTAs of H threads that fill 1024 threads of an SM (at most 32 CTAs).
constexpr int col_min_blocks(int H) { return 1024 / H > 32 ? 32 : (1024 / H > 0 ? 1024 / H : 1); }

template <int H>
__global__ void __launch_bounds__(H) k_fcol_fwd(const float2* __restrict__ in, float2* __restrict__ out, int Wh,
                                                int Whp, const float2* __restrict__ twH) {
  extern __shared__ float2 sm[];
  float2* tw = sm;  // per-pass twiddles
  float2* b0 = sm + reg::Passes<H>::TWSIZE;
  float2* b1 = b0 + reg::batch_rows(H) * kS;
  const int b = threadIdx.x & 7, tt = threadIdx.x >> 3;
  const int col = blockIdx.x * kB + b;
  const bool ok = col < Wh;
  const float2* src = in + static_cast<size_t>(H) * Wh * blockIdx.y + col;
  float2 v[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = ok ? src[static_cast<size_t>(tt + k * (H / 8)) * Wh] : make_float2(0.f, 0.f);
  load_pass_table<H, 1>(tw, twH);
  __syncthreads();
  reg::fft<H, -1>(v, tt, b, b0, b1, tw);
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

// Analysis fan-out: for every item (tile, filter) of the CTA's range,
// Y_f = column-inverse(W_f * uhat) on the tile.  The next item's filter tile
// (and, at a tile change, the next spectrum tile) is requested while the
// current transform runs.
template <int H>
__global__ void __launch_bounds__(H, col_min_blocks(H))
    k_fcol_fan(const float2* __restrict__ uhat, const float* __restrict__ bank, const WorkItem* __restrict__ items,
               const int* __restrict__ cta_begin, float2* __restrict__ Y, int Wh, int Whp, int label, int f0,
               const float2* __restrict__ twH) {
  extern __shared__ float2 sm[];
  float2* tw = sm;  // per-pass twiddles
  float2* b0 = sm + reg::Passes<H>::TWSIZE;
  float2* b1 = b0 + reg::batch_rows(H) * kS;
  const int ib = cta_begin[blockIdx.x], ie = cta_begin[blockIdx.x + 1];
  if (ib >= ie) return;
  const int b = threadIdx.x & 7, tt = threadIdx.x >> 3;
  const size_t Pb = static_cast<size_t>(H) * Wh, Pp = static_cast<size_t>(H) * Whp;
  WorkItem it = items[ib];
  int col = it.tile * kB + b;
  bool ok = col < Wh;
  float2 u[8];
  float w[8];
  load_tile8<H>(u, uhat + Pp * label, Whp, tt, col, ok);
  load_bank8<H>(w, bank + Pb * (f0 + it.filter), Wh, tt, col, ok);
  load_pass_table<H, 1>(tw, twH);
  __syncthreads();
  for (int i = ib; i < ie; ++i) {
    float2 v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = c_scale(u[k], w[k]);
    const int fl = it.filter, ccol = col;
    const bool cok = ok;
    if (i + 1 < ie) {
      const WorkItem nx = items[i + 1];
      col = nx.tile * kB + b;
      ok = col < Wh;
      load_bank8<H>(w, bank + Pb * (f0 + nx.filter), Wh, tt, col, ok);
      if (nx.tile != it.tile) load_tile8<H>(u, uhat + Pp * label, Whp, tt, col, ok);
      it = nx;
    }
    reg::fft<H, +1>(v, tt, b, b0, b1, tw);
    if (cok) {
      float2* dst = Y + Pp * fl + ccol;
#pragma unroll
      for (int k = 0; k < 8; ++k) dst[static_cast<size_t>(tt + k * (H / 8)) * Whp] = v[k];
    }
  }
}

// Synthesis gather: partial[label][slot] = sum over a run of items of one
// tile of W_f * column-forward(Y_f), stored compactly as [H][8]; the next
// item's coefficient tile is requested while the current transform runs.
template <int H>
__global__ void __launch_bounds__(H, col_min_blocks(H))
    k_fcol_gather(const float2* __restrict__ Y, const float* __restrict__ bank, const WorkItem* __restrict__ items,
                  const int* __restrict__ cta_begin, float2* __restrict__ partial, int Wh, int Whp, int nslots,
                  int label, int f0, const float2* __restrict__ twH) {
  extern __shared__ float2 sm[];
  float2* tw = sm;  // per-pass twiddles
  float2* b0 = sm + reg::Passes<H>::TWSIZE;
  float2* b1 = b0 + reg::batch_rows(H) * kS;
  const int ib = cta_begin[blockIdx.x], ie = cta_begin[blockIdx.x + 1];
  if (ib >= ie) return;
  const int b = threadIdx.x & 7, tt = threadIdx.x >> 3;
  const size_t Pb = static_cast<size_t>(H) * Wh, Pp = static_cast<size_t>(H) * Whp;
  WorkItem it = items[ib];
  int col = it.tile * kB + b;
  bool ok = col < Wh;
  float2 acc[8], y[8];
  float w[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) acc[k] = make_float2(0.f, 0.f);
  load_tile8<H>(y, Y + Pp * it.filter, Whp, tt, col, ok);
  load_pass_table<H, 1>(tw, twH);
  __syncthreads();
  for (int i = ib; i < ie; ++i) {
    float2 v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = y[k];
    load_bank8<H>(w, bank + Pb * (f0 + it.filter), Wh, tt, col, ok);
    WorkItem nx = it;
    int ncol = col;
    bool nok = ok;
    if (i + 1 < ie) {
      nx = items[i + 1];
      ncol = nx.tile * kB + b;
      nok = ncol < Wh;
      load_tile8<H>(y, Y + Pp * nx.filter, Whp, tt, ncol, nok);
    }
    reg::fft<H, -1>(v, tt, b, b0, b1, tw);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      acc[k].x = fmaf(w[k], v[k].x, acc[k].x);
      acc[k].y = fmaf(w[k], v[k].y, acc[k].y);
    }
    if (i + 1 == ie || nx.slot != it.slot) {
      float2* dst = partial + (static_cast<size_t>(label) * nslots + it.slot) * H * kB + b;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        dst[static_cast<size_t>(tt + k * (H / 8)) * kB] = acc[k];
        acc[k] = make_float2(0.f, 0.f);
      }
    }
    it = nx;
    col = ncol;
    ok = nok;
  }
}

// T[label] on one tile = column-inverse of the sum of the tile's partial
// slots, in the fixed slot order (filter order).
template <int H>
__global__ void __launch_bounds__(H) k_fcol_reduce_inv(const float2* __restrict__ partial,
                                                       const int* __restrict__ tile_begin,
                                                       const int* __restrict__ tile_slots, float2* __restrict__ T,
                                                       int Wh, int nslots, const float2* __restrict__ twH) {
  extern __shared__ float2 sm[];
  float2* tw = sm;  // per-pass twiddles
  float2* b0 = sm + reg::Passes<H>::TWSIZE;
  float2* b1 = b0 + reg::batch_rows(H) * kS;
  const int b = threadIdx.x & 7, tt = threadIdx.x >> 3;
  const int tile = blockIdx.x, label = blockIdx.y;
  const int col = tile * kB + b;
  const bool ok = col < Wh;
  float2 v[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = make_float2(0.f, 0.f);
  const int s0 = tile_begin[tile], s1 = tile_begin[tile + 1];
  for (int si = s0; si < s1; ++si) {
    const float2* src = partial + (static_cast<size_t>(label) * nslots + tile_slots[si]) * H * kB + b;
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = c_add(v[k], src[static_cast<size_t>(tt + k * (H / 8)) * kB]);
  }
  load_pass_table<H, 1>(tw, twH);
  __syncthreads();
  reg::fft<H, +1>(v, tt, b, b0, b1, tw);
  if (ok) {
    float2* dst = T + static_cast<size_t>(H) * Wh * label + col;
#pragma unroll
    for (int k = 0; k < 8; ++k) dst[static_cast<size_t>(tt + k * (H / 8)) * Wh] = v[k];
  }
}

// ---------------------------------------------------------------------------
// Row kernels: a real row of length W = 2L is the complex row
// z[n] = x[2n] + i x[2n+1], transformed by a group of T = L/8 threads.
// ---------------------------------------------------------------------------

// 16-byte asynchronous copies global -> shared (the copying thread waits for
// its own copies with cp_async_wait_all; the group barrier then publishes
// them to the group).  `evict_first`: the source is streamed through L2.
__device__ __forceinline__ void cp_async16(void* dst_smem, const void* src, bool evict_first, uint64_t policy) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst_smem));
  if (evict_first)
    asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "l"(policy)
                 : "memory");
  else
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ uint64_t evict_first_policy() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// Shared memory of one row group of k_wrow_shrink: FFT exchange buffer(s),
// and the stage that receives the next row's spectrum columns and b_v row.
// Every region is a whole number of 16-byte units (even float2 counts) so that
// the stage is 16-byte aligned for the asynchronous copies.
__host__ __device__ constexpr int even2(int n) { return (n + 1) & ~1; }
template <int L>
struct RowGroupSmem {
  static constexpr int T = L / 8;
  static constexpr int NBUF = T <= 32 ? 1 : 2;  // warp-sized groups exchange through one buffer
  static constexpr int BUF = even2(reg::row_buf(L));
  static constexpr int SX = L + 8;              // spectrum columns [c0, c0 + SX), SX >= the row pitch
  static constexpr int SB = L;                  // b_v row as float2
  static constexpr int SIZE = NBUF * BUF + SX + SB;
  static constexpr int TW = even2(L + 1);                     // exp(-2 pi i m / W), m <= L
  static constexpr int PT = even2(reg::Passes<L>::TWSIZE);    // per-pass twiddles
  static constexpr int RPC = 256 / T;                         // row groups per CTA of 256 threads
  static constexpr int TOTAL = TW + PT + RPC * SIZE;          // float2 per CTA
};

// v-step and b_v update of Sec. 3 on rows of (S u)_f: g = b_v + c,
// b_v <- clip(g, -t, t), d = soft(g, t) - clip(g, -t, t) = g - 2 clip(g);
// d (= v - b_v of the new iterate) is transformed back in place.
// Rows r = (filter fl, row) with r = fl H + row over the wave's nf filters;
// resident CTAs, each row group takes rows gid, gid + G, ... (G groups in
// all).  While a group transforms its row, the next row's spectrum columns
// (only the filter's column tiles [c0, c1]) and b_v row are copied into the
// group's stage; the twiddle tables are built once per CTA.
template <int L>
__global__ void __launch_bounds__(256, 4) k_wrow_shrink(float2* __restrict__ Y, float* __restrict__ bv,
                                                        const float* __restrict__ thr,
                                                        const int2* __restrict__ ranges, int H, int Whp, int eta,
                                                        int label, int f0, int nf, float scale,
                                                        const float2* __restrict__ twW) {
  using SM = RowGroupSmem<L>;
  constexpr int T = SM::T;
  constexpr int RPC = SM::RPC;
  extern __shared__ __align__(16) float2 sm[];
  float2* tw = sm;                    // exp(-2 pi i m / W), m <= L
  float2* pt = tw + SM::TW;           // per-pass twiddles of the length-L transform
  const int grp = threadIdx.x / T, tt = threadIdx.x % T;
  float2* gb = pt + SM::PT + grp * SM::SIZE;
  float2* fb0 = gb;
  float2* fb1 = gb + (SM::NBUF - 1) * SM::BUF;
  float2* sX = gb + SM::NBUF * SM::BUF;
  float2* sB = sX + SM::SX;
  const int bar = 1 + grp;
  const int G = gridDim.x * RPC;
  const int gid = blockIdx.x * RPC + grp;
  const int rows = nf * H;
  const int niter = (rows + G - 1) / G;  // the same for every group: dead rows still take part in barriers
  const uint64_t pol = evict_first_policy();

  // request row r's spectrum columns (its filter's column range only) and
  // its b_v row into the stage
  auto request_x = [&](int r) {
    if (r >= rows) return;
    const int fl = r / H, row = r - fl * H;
    const int2 rg = ranges[f0 + fl];
    if (rg.x <= rg.y) {
      const int c0 = rg.x & ~7;
      const int c1e = min(Whp, (rg.y | 7) + 1);
      const float2* X = Y + (static_cast<size_t>(fl) * H + row) * Whp + c0;
      for (int q = tt; q < (c1e - c0) / 2; q += T) cp_async16(sX + 2 * q, X + 2 * q, false, pol);
    }
  };
  auto request_b = [&](int r) {
    if (r >= rows) return;
    const int fl = r / H, row = r - fl * H;
    const float2* B =
        reinterpret_cast<const float2*>(bv) + ((static_cast<size_t>(label) * eta + f0 + fl) * H + row) * L;
    for (int q = tt; q < L / 2; q += T) cp_async16(sB + 2 * q, B + 2 * q, true, pol);
  };

  request_x(gid);
  request_b(gid);
  load_table(tw, twW, L + 1);
  reg::build_pass_twiddles<L, 2>(pt, twW, threadIdx.x, blockDim.x);
  __syncthreads();
  for (int it = 0; it < niter; ++it) {
    const int r = gid + it * G;
    const bool live = r < rows;
    const int fl = live ? r / H : 0, row = live ? r - fl * H : 0, f = f0 + fl;
    const int2 rg = ranges[f];
    const bool any = live && rg.x <= rg.y;
    const int c0 = any ? (rg.x & ~7) : L + 1;
    const int c1 = any ? min(L, (rg.y | 7)) : -1;
    const float th = thr[f];
    cp_async_commit_wait_all();
    reg::group_sync<T>(bar);
    float2 v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {  // inverse packing Z[n] = (X_n + conj X_{L-n}) + i e^{+2 pi i n/W} (X_n - conj X_{L-n})
      const int n = tt + k * T, m = L - n;
      const float2 a = (n >= c0 && n <= c1) ? sX[n - c0] : make_float2(0.f, 0.f);
      const float2 c = (m >= c0 && m <= c1) ? c_conj(sX[m - c0]) : make_float2(0.f, 0.f);
      const float2 s2 = c_add(a, c), d = c_sub(a, c);
      const float2 t = c_mul(c_conj(tw[n]), d);
      v[k] = make_float2(s2.x - t.y, s2.y + t.x);
    }
    reg::group_sync<T>(bar);  // the spectrum stage is read: refill it with the group's next row
    request_x(r + G);
    if (SM::NBUF == 1)
      reg::row_fft1<L, +1>(v, tt, fb0, pt, bar);
    else
      reg::row_fft<L, +1>(v, tt, fb0, fb1, pt, bar);
    float2* X = Y + (static_cast<size_t>(fl) * H + row) * Whp;
    if (live) {
      float2* b2 = reinterpret_cast<float2*>(bv) + ((static_cast<size_t>(label) * eta + f) * H + row) * L;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const float2 bo = sB[tt + k * T];
        const float gx = fmaf(scale, v[k].x, bo.x), gy = fmaf(scale, v[k].y, bo.y);
        const float cx = fminf(fmaxf(gx, -th), th), cy = fminf(fmaxf(gy, -th), th);
        __stcs(b2 + tt + k * T, make_float2(cx, cy));
        v[k] = make_float2(gx - 2.f * cx, gy - 2.f * cy);
      }
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = make_float2(0.f, 0.f);
    }
    reg::group_sync<T>(bar);  // the b_v stage is read: refill it with the group's next row
    request_b(r + G);
    if (SM::NBUF == 1)
      reg::row_fft1<L, -1>(v, tt, fb0, pt, bar);
    else
      reg::row_fft<L, -1>(v, tt, fb0, fb1, pt, bar);
    float2* ub = SM::NBUF == 1 ? fb0 : fb1;
    reg::group_sync<T>(bar);  // the last pass may still read the buffer
#pragma unroll
    for (int k = 0; k < 8; ++k) ub[reg::ridx(tt + k * T)] = v[k];
    reg::group_sync<T>(bar);
    // forward unpacking X[k] = 1/2 [(Z_k + conj Z_{L-k}) - i e^{-2 pi i k/W} (Z_k - conj Z_{L-k})]
    for (int i = c0 + tt; i <= c1; i += T) {
      const float2 a = ub[reg::ridx(i == L ? 0 : i)];
      const float2 c = c_conj(ub[reg::ridx(i == 0 ? 0 : L - i)]);
      const float2 s2 = c_add(a, c), d = c_sub(a, c);
      const float2 t = c_mul(tw[i], d);
      X[i] = make_float2(0.5f * (s2.x + t.y), 0.5f * (s2.y - t.x));
    }
  }
  cp_async_commit_wait_all();  // no copy outlives the kernel
}

// Euclidean projection of g[0..K) onto the unit simplex, as the paper
// constructs it: project onto the hyperplane sum = 1 (g + (1 - sum g)/q), set
// the negative components to zero and repeat on the remaining ones (at most K
// passes; the result is exact).
template <int KMAX>
__device__ __forceinline__ void simplex_project(float (&g)[KMAX], int K) {
  unsigned act = (1u << K) - 1u;
  float tau = 0.f;
  for (int pass = 0; pass < K; ++pass) {
    float sum = 0.f;
    int q = 0;
#pragma unroll
    for (int k = 0; k < KMAX; ++k)
      if ((act >> k) & 1u) {
        sum += g[k];
        ++q;
      }
    tau = (sum - 1.f) / static_cast<float>(q);
    unsigned nact = act;
#pragma unroll
    for (int k = 0; k < KMAX; ++k)
      if (((act >> k) & 1u) && g[k] - tau < 0.f) nact &= ~(1u << k);
    if (nact == act) break;
    act = nact;
  }
#pragma unroll
  for (int k = 0; k < KMAX; ++k) g[k] = ((act >> k) & 1u) ? g[k] - tau : 0.f;
}

// u-step (u = 1/2 [S^T(v - b_v) + (w - b_w) - gamma s], A^T A = 2I), w-step
// (pixelwise simplex projection of g_w = b_w + u), b_w = g_w - w, and the row
// spectra of u for the next analysis.  One row per group of L/8 threads, all
// K labels; the carried values of a thread live in its private slots of U.
template <int L, int KMAX>
__global__ void __launch_bounds__(256) k_wrow_ustep(const float2* __restrict__ Tsp, const float* __restrict__ s,
                                                    float* __restrict__ w, float* __restrict__ bw,
                                                    float* __restrict__ u, float2* __restrict__ Ur, int K, int H,
                                                    float scale, float gamma, const float2* __restrict__ twW) {
  constexpr int T = L / 8;
  constexpr int RPC = 256 / T;
  constexpr int BUF = reg::row_buf(L);
  constexpr int Wh = L + 1;
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* pt = tw + (L + 1);
  const int grp = threadIdx.x / T, tt = threadIdx.x % T;
  float2* b0 = pt + reg::Passes<L>::TWSIZE + grp * 2 * BUF;
  float2* b1 = b0 + BUF;
  float2* U = pt + reg::Passes<L>::TWSIZE + RPC * 2 * BUF;  // [k][e][thread]
  const int bar = 1 + grp;
  const int row = blockIdx.x * RPC + grp;
  const bool live = row < H;
  const int rowc = live ? row : 0;
  const size_t HL = static_cast<size_t>(H) * L, HWh = static_cast<size_t>(H) * Wh;
  auto slot = [&](int k, int e) { return (k * 8 + e) * 256 + threadIdx.x; };
  load_table(tw, twW, L + 1);
  reg::build_pass_twiddles<L, 2>(pt, twW, threadIdx.x, blockDim.x);
  __syncthreads();
  // S^T(v - b_v) on this row, label by label
  for (int k = 0; k < K; ++k) {
    reg::group_sync<T>(bar);  // the previous label's transform may still read b1
    const float2* X = Tsp + HWh * k + static_cast<size_t>(rowc) * Wh;
    for (int i = tt; i <= L; i += T) b1[reg::ridx(i)] = live ? X[i] : make_float2(0.f, 0.f);
    reg::group_sync<T>(bar);
    float2 v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int n = tt + e * T;
      const float2 a = b1[reg::ridx(n)];
      const float2 c = c_conj(b1[reg::ridx(L - n)]);
      const float2 sm2 = c_add(a, c), d = c_sub(a, c);
      const float2 t = c_mul(c_conj(tw[n]), d);
      v[e] = make_float2(sm2.x - t.y, sm2.y + t.x);
    }
    reg::row_fft<L, +1>(v, tt, b0, b1, pt, bar);
#pragma unroll
    for (int e = 0; e < 8; ++e) U[slot(k, e)] = c_scale(v[e], scale);
  }
  // pointwise u-step, projection and b_w update (two pixels per slot)
  if (live) {
    const float2* s2 = reinterpret_cast<const float2*>(s) + static_cast<size_t>(row) * L;
    float2* w2 = reinterpret_cast<float2*>(w) + static_cast<size_t>(row) * L;
    float2* bw2 = reinterpret_cast<float2*>(bw) + static_cast<size_t>(row) * L;
    float2* u2 = reinterpret_cast<float2*>(u) + static_cast<size_t>(row) * L;
    const float hg = 0.5f * gamma;
#pragma unroll 1
    for (int e = 0; e < 8; ++e) {
      const int n = tt + e * T;
      float gx[KMAX], gy[KMAX];
#pragma unroll
      for (int k = 0; k < KMAX; ++k) {
        gx[k] = 0.f;
        gy[k] = 0.f;
        if (k < K) {
          const float2 st = U[slot(k, e)];
          const float2 wv = w2[HL * k + n], bv = bw2[HL * k + n], sv = s2[HL * k + n];
          const float ux = 0.5f * (st.x + (wv.x - bv.x)) - hg * sv.x;
          const float uy = 0.5f * (st.y + (wv.y - bv.y)) - hg * sv.y;
          u2[HL * k + n] = make_float2(ux, uy);
          U[slot(k, e)] = make_float2(ux, uy);
          gx[k] = bv.x + ux;
          gy[k] = bv.y + uy;
        }
      }
      float px[KMAX], py[KMAX];
#pragma unroll
      for (int k = 0; k < KMAX; ++k) {
        px[k] = gx[k];
        py[k] = gy[k];
      }
      simplex_project<KMAX>(px, K);
      simplex_project<KMAX>(py, K);
#pragma unroll
      for (int k = 0; k < KMAX; ++k)
        if (k < K) {
          w2[HL * k + n] = make_float2(px[k], py[k]);
          bw2[HL * k + n] = make_float2(gx[k] - px[k], gy[k] - py[k]);
        }
    }
  } else {
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int e = 0; e < 8; ++e) U[slot(k, e)] = make_float2(0.f, 0.f);
  }
  // row spectra of u
  for (int k = 0; k < K; ++k) {
    float2 v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = U[slot(k, e)];
    reg::row_fft<L, -1>(v, tt, b0, b1, pt, bar);
    reg::group_sync<T>(bar);
#pragma unroll
    for (int e = 0; e < 8; ++e) b1[reg::ridx(tt + e * T)] = v[e];
    reg::group_sync<T>(bar);
    if (live) {
      float2* X = Ur + HWh * k + static_cast<size_t>(row) * Wh;
      for (int i = tt; i <= L; i += T) {
        const float2 a = b1[reg::ridx(i == L ? 0 : i)];
        const float2 c = c_conj(b1[reg::ridx(i == 0 ? 0 : L - i)]);
        const float2 sm2 = c_add(a, c), d = c_sub(a, c);
        const float2 t = c_mul(tw[i], d);
        X[i] = make_float2(0.5f * (sm2.x + t.y), 0.5f * (sm2.y - t.x));
      }
    }
  }
}

template <int L>
size_t ustep_smem(int K) {
  return sizeof(float2) * ((L + 1) + reg::Passes<L>::TWSIZE + (256 / (L / 8)) * 2 * reg::row_buf(L) + K * 8 * 256);
}

template <int N>
size_t col_smem() {
  return sizeof(float2) * (reg::Passes<N>::TWSIZE + 2 * reg::batch_rows(N) * kS);
}

template <int L>
size_t shrink_smem() {
  return sizeof(float2) * RowGroupSmem<L>::TOTAL;
}

template <int L>
size_t row_smem() {
  return sizeof(float2) * ((L + 1) + reg::Passes<L>::TWSIZE + (256 / (L / 8)) * 2 * reg::row_buf(L));
}

template <int L>
int row_rows_per_cta() {
  return 256 / (L / 8);
}

template <int H, int L>
cudaError_t iteration_body(const Geo& g, const FastPlan& plan, const float2* Ur, float2* uhat, float2* Y, float* bv,
                           const float* thr, float2* partial, float2* T, int K, float scale, cudaStream_t st,
                           const LaunchHook& hook) {
  const int ntiles = (g.Wh + kB - 1) / kB;
  const int Whp = fast_pitch(g);
  const int nslots = plan.nslots;
  const int nw = static_cast<int>(plan.wave_f0.size());
  hook.mark(kKindColFwd);
  k_fcol_fwd<H><<<dim3(ntiles, K), H, col_smem<H>(), st>>>(Ur, uhat, g.Wh, Whp, g.twH);
  for (int label = 0; label < K; ++label) {
    for (int w = 0; w < nw; ++w) {
      const int f0 = plan.wave_f0[w], nf = plan.wave_nf[w];
      const int c0 = plan.wave_cta0[w], nc = plan.wave_cta0[w + 1] - c0;
      const int* cb = plan.cta_begin + c0 + w;  // each wave's ranges end with one extra entry
      if (nc > 0) {
        hook.mark(kKindFan);
        k_fcol_fan<H><<<nc, H, col_smem<H>(), st>>>(uhat, g.bank, plan.items, cb, Y, g.Wh, Whp, label, f0, g.twH);
      }
      hook.mark(kKindShrink);
      {
        const int groups = (nf * g.H + RowGroupSmem<L>::RPC - 1) / RowGroupSmem<L>::RPC;
        const int ctas = std::min(groups, std::max(plan.row_ctas, 1));
        k_wrow_shrink<L><<<ctas, 256, shrink_smem<L>(), st>>>(Y, bv, thr, g.ranges, g.H, Whp, g.eta, label, f0, nf,
                                                              scale, g.twW);
      }
      if (nc > 0) {
        hook.mark(kKindGather);
        k_fcol_gather<H><<<nc, H, col_smem<H>(), st>>>(Y, g.bank, plan.items, cb, partial, g.Wh, Whp, nslots,
                                                        label, f0, g.twH);
      }
    }
  }
  hook.mark(kKindReduce);
  k_fcol_reduce_inv<H><<<dim3(ntiles, K), H, col_smem<H>(), st>>>(partial, plan.tile_begin, plan.tile_slots, T,
                                                                  g.Wh, nslots, g.twH);
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
  cudaError_t e = allow_smem(k_wrow_shrink<L>, shrink_smem<L>());
  if (e == cudaSuccess) e = allow_smem(k_wrow_ustep<L, 4>, ustep_smem<L>(4));
  if (e == cudaSuccess) e = allow_smem(k_wrow_ustep<L, 8>, ustep_smem<L>(8));
  return e;
}

template <int L>
cudaError_t ustep_launch(const Geo& g, const float2* T, const float* s, float* w, float* bw, float* u, float2* Ur,
                         int K, float gamma, float scale, cudaStream_t st) {
  constexpr int RPC = 256 / (L / 8);
  const dim3 grid((g.H + RPC - 1) / RPC);
  if (K <= 4)
    k_wrow_ustep<L, 4><<<grid, 256, ustep_smem<L>(K), st>>>(T, s, w, bw, u, Ur, K, g.H, scale, gamma, g.twW);
  else
    k_wrow_ustep<L, 8><<<grid, 256, ustep_smem<L>(K), st>>>(T, s, w, bw, u, Ur, K, g.H, scale, gamma, g.twW);
  return cudaGetLastError();
}

template <int H>
cudaError_t dispatch_L(const Geo& g, const FastPlan& plan, const float2* Ur, float2* uhat, float2* Y, float* bv,
                       const float* thr, float2* partial, float2* T, int K, float scale, cudaStream_t st,
                       const LaunchHook& hook) {
  switch (g.L) {
    case 8: return iteration_body<H, 8>(g, plan, Ur, uhat, Y, bv, thr, partial, T, K, scale, st, hook);
    case 16: return iteration_body<H, 16>(g, plan, Ur, uhat, Y, bv, thr, partial, T, K, scale, st, hook);
    case 32: return iteration_body<H, 32>(g, plan, Ur, uhat, Y, bv, thr, partial, T, K, scale, st, hook);
    case 64: return iteration_body<H, 64>(g, plan, Ur, uhat, Y, bv, thr, partial, T, K, scale, st, hook);
    case 128: return iteration_body<H, 128>(g, plan, Ur, uhat, Y, bv, thr, partial, T, K, scale, st, hook);
    case 256: return iteration_body<H, 256>(g, plan, Ur, uhat, Y, bv, thr, partial, T, K, scale, st, hook);
    case 512: return iteration_body<H, 512>(g, plan, Ur, uhat, Y, bv, thr, partial, T, K, scale, st, hook);
    case 1024: return iteration_body<H, 1024>(g, plan, Ur, uhat, Y, bv, thr, partial, T, K, scale, st, hook);
    default: return cudaErrorInvalidValue;
  }
}

bool pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

}  // namespace

int fast_pitch(const Geo& g) { return (g.Wh + 7) & ~7; }

bool fast_ustep_ok(const Geo& g, int K) {
  if (!fast_path_ok(g) || K > 8) return false;
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return false;
  size_t need = 0;
  switch (g.L) {
    case 8: need = ustep_smem<8>(K); break;
    case 16: need = ustep_smem<16>(K); break;
    case 32: need = ustep_smem<32>(K); break;
    case 64: need = ustep_smem<64>(K); break;
    case 128: need = ustep_smem<128>(K); break;
    case 256: need = ustep_smem<256>(K); break;
    case 512: need = ustep_smem<512>(K); break;
    case 1024: need = ustep_smem<1024>(K); break;
    default: return false;
  }
  return need <= static_cast<size_t>(optin);
}

cudaError_t run_fast_ustep(const Geo& g, const float2* T, const float* s, float* w, float* bw, float* u, float2* Ur,
                           int K, float gamma, float scale, cudaStream_t st) {
  switch (g.L) {
    case 8: return ustep_launch<8>(g, T, s, w, bw, u, Ur, K, gamma, scale, st);
    case 16: return ustep_launch<16>(g, T, s, w, bw, u, Ur, K, gamma, scale, st);
    case 32: return ustep_launch<32>(g, T, s, w, bw, u, Ur, K, gamma, scale, st);
    case 64: return ustep_launch<64>(g, T, s, w, bw, u, Ur, K, gamma, scale, st);
    case 128: return ustep_launch<128>(g, T, s, w, bw, u, Ur, K, gamma, scale, st);
    case 256: return ustep_launch<256>(g, T, s, w, bw, u, Ur, K, gamma, scale, st);
    case 512: return ustep_launch<512>(g, T, s, w, bw, u, Ur, K, gamma, scale, st);
    case 1024: return ustep_launch<1024>(g, T, s, w, bw, u, Ur, K, gamma, scale, st);
    default: return cudaErrorInvalidValue;
  }
}

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

int fast_wave(const Geo& g, int wave_mib) {
  // filters per wave: keep the wave's coefficient spectra near wave_mib MiB
  const size_t plane = sizeof(float2) * static_cast<size_t>(g.H) * fast_pitch(g);
  int w = static_cast<int>((static_cast<size_t>(wave_mib) << 20) / plane);
  if (w < 1) w = 1;
  if (w > g.eta) w = g.eta;
  // balance the waves of a label
  const int nw = (g.eta + w - 1) / w;
  return (g.eta + nw - 1) / nw;
}

int fast_col_ctas(const Geo& g, int per_sm) {
  int dev = 0, sms = 0, fit = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  cudaError_t e = cudaErrorInvalidValue;
  switch (g.H) {
#define SHF_OCC(HH)                                                                                   \
  case HH:                                                                                            \
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, k_fcol_gather<HH>, HH, col_smem<HH>()); \
    break;
    SHF_OCC(8) SHF_OCC(16) SHF_OCC(32) SHF_OCC(64) SHF_OCC(128) SHF_OCC(256) SHF_OCC(512) SHF_OCC(1024)
#undef SHF_OCC
    default: break;
  }
  if (e != cudaSuccess || fit < 1) return 0;
  const int k = (per_sm <= 0 || per_sm > fit) ? fit : per_sm;
  return k * sms;
}

int fast_row_ctas(const Geo& g) {
  int dev = 0, sms = 0, fit = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  cudaError_t e = cudaErrorInvalidValue;
  switch (g.L) {
#define SHF_OCC(LL)                                                                                          \
  case LL:                                                                                                   \
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, k_wrow_shrink<LL>, 256, shrink_smem<LL>()); \
    break;
    SHF_OCC(8) SHF_OCC(16) SHF_OCC(32) SHF_OCC(64) SHF_OCC(128) SHF_OCC(256) SHF_OCC(512) SHF_OCC(1024)
#undef SHF_OCC
    default: break;
  }
  if (e != cudaSuccess || fit < 1) return 0;
  return fit * sms;
}

void build_fast_plan(const Geo& g, const int2* ranges, FastPlan* plan, std::vector<WorkItem>* items,
                     std::vector<int>* cta_begin, std::vector<int>* tile_begin, std::vector<int>* tile_slots) {
  const int ntiles = (g.Wh + kB - 1) / kB;
  const int wave = fast_wave(g, plan->wave_mib);
  const int ctas = plan->col_ctas > 0 ? plan->col_ctas : 1;
  items->clear();
  cta_begin->clear();
  plan->wave_f0.clear();
  plan->wave_nf.clear();
  plan->wave_cta0.clear();
  std::vector<std::vector<int>> per_tile(ntiles);
  int slot = 0;
  for (int f0 = 0; f0 < g.eta; f0 += wave) {
    const int nf = std::min(wave, g.eta - f0);
    plan->wave_f0.push_back(f0);
    plan->wave_nf.push_back(nf);
    // this wave's (tile, filter) pairs in (tile, filter) order
    const size_t first = items->size();
    for (int t = 0; t < ntiles; ++t)
      for (int fl = 0; fl < nf; ++fl) {
        const int2 r = ranges[f0 + fl];
        if (r.x <= r.y && t >= (r.x >> 3) && t <= (r.y >> 3)) items->push_back(WorkItem{t, fl, 0, 0});
      }
    const long n = static_cast<long>(items->size() - first);
    const int G = static_cast<int>(std::min<long>(ctas, n));
    plan->wave_cta0.push_back(static_cast<int>(cta_begin->size()) - static_cast<int>(plan->wave_cta0.size()));
    for (int c = 0; c <= G; ++c) cta_begin->push_back(static_cast<int>(first + (G > 0 ? n * c / G : 0)));
    // one partial slot per run of one tile inside a CTA's range
    for (int c = 0; c < G; ++c) {
      const long b = n * c / G, e = n * (c + 1) / G;
      for (long i = b; i < e; ++i) {
        WorkItem& it = (*items)[first + i];
        if (i == b || (*items)[first + i - 1].tile != it.tile) per_tile[it.tile].push_back(slot++);
        it.slot = slot - 1;
      }
    }
  }
  plan->wave_cta0.push_back(static_cast<int>(cta_begin->size()) - static_cast<int>(plan->wave_cta0.size()));
  plan->nslots = slot;
  tile_begin->assign(1, 0);
  tile_slots->clear();
  for (int t = 0; t < ntiles; ++t) {
    for (int sl : per_tile[t]) tile_slots->push_back(sl);
    tile_begin->push_back(static_cast<int>(tile_slots->size()));
  }
  if (items->empty()) items->push_back(WorkItem{0, 0, 0, 0});  // keep the device arrays non-empty
  if (tile_slots->empty()) tile_slots->push_back(0);
}

cudaError_t run_fast_iteration_body(const Geo& g, const FastPlan& plan, const float2* Ur, float2* uhat, float2* Y,
                                    float* bv, const float* thr, float2* partial, float2* T, int K, float scale,
                                    cudaStream_t st, const LaunchHook& hook) {
  switch (g.H) {
    case 8: return dispatch_L<8>(g, plan, Ur, uhat, Y, bv, thr, partial, T, K, scale, st, hook);
    case 16: return dispatch_L<16>(g, plan, Ur, uhat, Y, bv, thr, partial, T, K, scale, st, hook);
    case 32: return dispatch_L<32>(g, plan, Ur, uhat, Y, bv, thr, partial, T, K, scale, st, hook);
    case 64: return dispatch_L<64>(g, plan, Ur, uhat, Y, bv, thr, partial, T, K, scale, st, hook);
    case 128: return dispatch_L<128>(g, plan, Ur, uhat, Y, bv, thr, partial, T, K, scale, st, hook);
    case 256: return dispatch_L<256>(g, plan, Ur, uhat, Y, bv, thr, partial, T, K, scale, st, hook);
    case 512: return dispatch_L<512>(g, plan, Ur, uhat, Y, bv, thr, partial, T, K, scale, st, hook);
    case 1024: return dispatch_L<1024>(g, plan, Ur, uhat, Y, bv, thr, partial, T, K, scale, st, hook);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace shf

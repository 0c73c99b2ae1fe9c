// Row transforms of the fast path: the v-step (soft shrinkage and b_v update
// between the inverse and forward row transforms of every coefficient row)
// and the u/w-step (Sec. 3).
#include <algorithm>

#include "shf_fast.h"
#include "shf_fft16.cuh"
#include "shf_fftv.cuh"
#include "shf_simplex.cuh"

namespace shf {
namespace fast {
namespace {

// Row groups of T = L/8 threads inside CTAs of NTH threads.  When T divides
// 32 a warp holds 32/T groups; when T is a multiple of 32 a group is T/32
// whole warps (their barriers stay inside the group).  Otherwise (T = 3 2^a
// or 5 2^a, a < 5) the groups are packed back to back over CTAs of a multiple
// of lcm(T, 32) = 32 R threads, every lane busy, and the group barrier is the
// CTA's.  Lanes that a layout leaves idle mirror a lane of a real group (same
// shared-memory values) and write nothing to global memory.
template <int L>
struct RowGeo {
  static constexpr int T = L / 8;
  static constexpr bool TILE = reg::tiles_warps(T);
  static constexpr int LCM = 32 * reg::odd_part(T);        // lcm(T, 32) when !TILE
  static constexpr int GPW = T <= 32 ? 32 / T : 1;         // groups per warp
  static constexpr int WPG = T <= 32 ? 1 : (T + 31) / 32;  // warps per group
  static constexpr int NTH = TILE ? (T <= 32 ? 256 : (8 / WPG) * WPG * 32) : (256 / LCM > 0 ? 256 / LCM : 1) * LCM;
  static constexpr int RPC = TILE ? (T <= 32 ? 8 * GPW : 8 / WPG) : NTH / T;  // groups per CTA
  __device__ static void locate(int& grp, int& tt, bool& act) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (!TILE) {
      grp = threadIdx.x / T;
      tt = threadIdx.x - grp * T;
      act = true;
    } else if (T <= 32) {
      const int g = lane / T;
      act = g < GPW;
      grp = warp * GPW + (act ? g : GPW - 1);
      tt = act ? lane - g * T : T - 1;
    } else {
      grp = warp / WPG;
      tt = (warp % WPG) * 32 + lane;
      act = tt < T;
      if (!act) tt = T - 1;
    }
  }
};

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

// Shared memory of one row group of the v-step kernels: FFT exchange
// buffer(s), and the stage that receives the next row's spectrum columns and
// b_v row (the adjoint also its coefficient codes, and a slot per thread for
// the row's threshold sum).  Every region is a whole number of 16-byte units
// (even float2 counts) so that the stage is 16-byte aligned for the
// asynchronous copies.
__host__ __device__ constexpr int even2(int n) { return (n + 1) & ~1; }
template <int L, int MODE>
struct RowGroupSmem {
  static constexpr int T = L / 8;
  static constexpr int NBUF = T <= 32 ? 1 : 2;  // warp-sized groups exchange through one buffer
  static constexpr int BUF = even2(reg::row_buf(L));
  static constexpr int SX = L + 8;              // spectrum columns [c0, c0 + SX), SX >= the row pitch
  static constexpr int SB = L;                  // b_v (or its adjoint) row as float2
  static constexpr int SC = MODE == 1 ? L / 4 : 0;        // codes of the row: 2L bytes
  static constexpr int SD = MODE == 1 ? even2(T) : 0;     // one double per thread
  static constexpr int SIZE = NBUF * BUF + SX + SB + SC + SD;
  static constexpr int TW = even2(L + 1);                     // exp(-2 pi i m / W), m <= L
  static constexpr int PT = even2(reg::Passes<L>::TWSIZE);    // per-pass twiddles
  static constexpr int RPC = RowGeo<L>::RPC;                  // row groups per CTA
  static constexpr int TOTAL = TW + PT + RPC * SIZE;          // float2 per CTA
};

// Code of a coefficient for the reverse mode: 0 where |g| < t (clip is the
// identity, soft shrinkage is 0), else the sign of g.
__device__ __forceinline__ signed char clip_code(float g, float t) {
  return fabsf(g) < t ? 0 : (g > 0.f ? 1 : -1);
}

// MODE 0: v-step and b_v update of Sec. 3 on rows of (S u)_f: g = b_v + c,
// b_v <- clip(g, -t, t), d = soft(g, t) - clip(g, -t, t) = g - 2 clip(g);
// d (= v - b_v of the new iterate) is transformed back in place.  With `code`
// non-null it also records clip_code(g, t) per coefficient.
// MODE 1: its adjoint for the reverse mode of the unrolled iteration: with
// dbar = c (the rows of S Qbar) and the recorded codes m,
// bvbar <- bvbar - dbar where m = 0, dbar elsewhere; the row's threshold sum
// sum m (bvbar - 2 dbar) over m != 0 (FP64, fixed order) goes to
// tpart[(label eta + f) H + row] (each thread sums its 16 terms in FP32 in a
// fixed order; the group's partials are added in FP64 in thread order); the
// new bvbar is transformed back in place (the input of S^T).
// Rows r = (pair fl, row) with r = fl H + row over the wave's nv (label,
// filter) pairs, fl = (label - l0) nf + (f - f0);
// resident CTAs, each row group takes rows gid, gid + G, ... (G groups in
// all).  While a group transforms its row, the next row's spectrum columns
// (only the filter's column tiles [c0, c1]) and b_v row are copied into the
// group's stage; the twiddle tables are built once per CTA.  Column ranges
// are widened to the column kernels' tiles (8 columns, or 4 for H > 1024).
// Four CTAs of 256 threads per SM (64 registers) for powers of two; three for
// L = 3 2^a or 5 2^a, whose radix-R pass holds more values.  The half widths
// 64..1024 take k_wrow_vstep16 instead (below); this kernel serves the others.
template <int L, int MODE>
__global__ void __launch_bounds__(RowGeo<L>::NTH, (reg::odd_part(L) == 1 ? 1024 : 768) / RowGeo<L>::NTH)
    k_wrow_vstep(float2* __restrict__ Y, float* __restrict__ bv, const float* __restrict__ thr,
                 const int2* __restrict__ ranges, int H, int Whp, int eta, int l0, int f0, int nf, int nv,
                 float scale, const float2* __restrict__ twW, signed char* __restrict__ code,
                 double* __restrict__ tpart) {
  using SM = RowGroupSmem<L, MODE>;
  constexpr int T = SM::T;
  constexpr int RPC = SM::RPC;
  extern __shared__ __align__(16) float2 sm[];
  float2* tw = sm;                    // exp(-2 pi i m / W), m <= L
  float2* pt = tw + SM::TW;           // per-pass twiddles of the length-L transform
  int grp, tt;
  bool act;
  RowGeo<L>::locate(grp, tt, act);
  float2* gb = pt + SM::PT + grp * SM::SIZE;
  float2* fb0 = gb;
  float2* fb1 = gb + (SM::NBUF - 1) * SM::BUF;
  float2* sX = gb + SM::NBUF * SM::BUF;
  float2* sB = sX + SM::SX;
  const char2* sC = reinterpret_cast<const char2*>(sB + SM::SB);
  double* sD = reinterpret_cast<double*>(sB + SM::SB + SM::SC);
  const int bar = 1 + grp;
  const int G = gridDim.x * RPC;
  const int gid = blockIdx.x * RPC + grp;
  const int rows = nv * H;
  const int niter = (rows + G - 1) / G;  // the same for every group: dead rows still take part in barriers
  // label and filter of pair fl
  auto pair_of = [&](int fl, int& lab, int& f) {
    const int q = fl / nf;
    lab = l0 + q;
    f = f0 + fl - q * nf;
  };
  const uint64_t pol = evict_first_policy();
  const size_t W = 2 * static_cast<size_t>(L);
  // the column kernels write whole tiles of reg::col_batch(H) columns: the
  // rows carry exactly those tiles
  const int cmask = reg::col_batch(H) - 1;
  // row r = fl H + row is tracked as (fl, row): one step of G rows adds
  // (gq, gr) with a carry, so the loop needs no division
  const int gq = G / H, gr = G - gq * H;
  auto advance = [&](int& fl, int& row) {
    fl += gq;
    row += gr;
    if (row >= H) {
      row -= H;
      ++fl;
    }
  };

  // request row (fl, row)'s spectrum columns (its filter's column range
  // only) and its b_v row (and codes) into the stage
  auto request_x = [&](int fl, int row) {
    if (fl >= nv || !act) return;
    int lab, f;
    pair_of(fl, lab, f);
    const int2 rg = ranges[f];
    if (rg.x <= rg.y) {
      const int c0 = rg.x & ~cmask;
      const int c1e = min(Whp, (rg.y | cmask) + 1);
      const float2* X = Y + (static_cast<size_t>(fl) * H + row) * Whp + c0;
      for (int q = tt; q < (c1e - c0) / 2; q += T) cp_async16(sX + 2 * q, X + 2 * q, false, pol);
    }
  };
  auto request_b = [&](int fl, int row) {
    if (fl >= nv || !act) return;
    int lab, f;
    pair_of(fl, lab, f);
    const size_t rix = (static_cast<size_t>(lab) * eta + f) * H + row;
    const float2* B = reinterpret_cast<const float2*>(bv) + rix * L;
    for (int q = tt; q < L / 2; q += T) cp_async16(sB + 2 * q, B + 2 * q, true, pol);
    if (MODE == 1) {  // 2L bytes of codes: L/8 = T chunks of 16 bytes
      const signed char* Cr = code + rix * W;
      cp_async16(sB + SM::SB + 2 * tt, Cr + 16 * tt, true, pol);
    }
  };

  // b_v was last written by this kernel's previous launch for the label,
  // which has completed: it may be requested before the wait
  int flc = gid / H, rowc = gid - flc * H;  // the group's current row
  request_b(flc, rowc);
  load_table(tw, twW, L + 1);
  reg::build_pass_twiddles<L, 2>(pt, twW, threadIdx.x, blockDim.x);
  pdl_wait();
  pdl_trigger();
  request_x(flc, rowc);
  __syncthreads();
  for (int it = 0; it < niter; ++it) {
    const bool live = flc < nv;
    const int fl = live ? flc : 0, row = live ? rowc : 0;
    int label, f;
    pair_of(fl, label, f);
    int fln = flc, rown = rowc;  // the group's next row
    advance(fln, rown);
    const int2 rg = ranges[f];
    const bool any = live && rg.x <= rg.y;
    const int c0 = any ? (rg.x & ~cmask) : L + 1;
    const int c1 = any ? min(L, (rg.y | cmask)) : -1;
    const float th = thr[f];
    const size_t rix = (static_cast<size_t>(label) * eta + f) * H + row;
    cp_async_commit_wait_all();
    reg::group_sync<T>(bar);
    float2 v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {  // inverse packing Z[n] = (X_n + conj X_{L-n}) + i e^{+2 pi i n/W} (X_n - conj X_{L-n})
      const int n = tt + k * T, m = L - n;
      const float2 a = (n >= c0 && n <= c1) ? sX[n - c0] : make_float2(0.f, 0.f);
      const float2 c = (m >= c0 && m <= c1) ? c_conj(sX[m - c0]) : make_float2(0.f, 0.f);
      const float2 s2 = c_add(a, c), d = c_sub(a, c);
      v[k] = pack_combine(s2, d, tw[n]);
    }
    reg::group_sync<T>(bar);  // the spectrum stage is read: refill it with the group's next row
    request_x(fln, rown);
    if (SM::NBUF == 1)
      reg::row_fft1<L, +1>(v, tt, fb0, pt, bar);
    else
      reg::row_fft<L, +1>(v, tt, fb0, fb1, pt, bar);
    float2* X = Y + (static_cast<size_t>(fl) * H + row) * Whp;
    if (live) {
      float2* b2 = reinterpret_cast<float2*>(bv) + rix * L;
      if (MODE == 0) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const float2 g = c_fma2(make_float2(scale, scale), v[k], sB[tt + k * T]);
          const float2 c = make_float2(fminf(fmaxf(g.x, -th), th), fminf(fmaxf(g.y, -th), th));
          if (act) __stcs(b2 + tt + k * T, c);
          if (code && act)
            reinterpret_cast<char2*>(code + rix * W)[tt + k * T] = make_char2(clip_code(g.x, th), clip_code(g.y, th));
          v[k] = c_fma2(make_float2(-2.f, -2.f), c, g);  // g - 2 clip(g)
        }
      } else {
        float tacc = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const float2 bo = sB[tt + k * T];
          const char2 m = sC[tt + k * T];
          const float dx = scale * v[k].x, dy = scale * v[k].y;
          const float nx = m.x == 0 ? bo.x - dx : dx;
          const float ny = m.y == 0 ? bo.y - dy : dy;
          tacc = fmaf(static_cast<float>(m.x), fmaf(-2.f, dx, bo.x), tacc);
          tacc = fmaf(static_cast<float>(m.y), fmaf(-2.f, dy, bo.y), tacc);
          if (act) __stcs(b2 + tt + k * T, make_float2(nx, ny));
          v[k] = make_float2(nx, ny);
        }
        sD[tt] = static_cast<double>(tacc);
      }
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = make_float2(0.f, 0.f);
    }
    reg::group_sync<T>(bar);  // the b_v stage is read: refill it with the group's next row
    if (MODE == 1 && live && act && tt == 0) {  // the row's threshold sum, in thread order
      double s = 0.0;
      for (int j = 0; j < T; ++j) s += sD[j];
      tpart[rix] = s;
    }
    request_b(fln, rown);
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
    // on columns i = c0 + tt + k T <= c1 (at most 9 per thread: L + 1 columns);
    // for T a multiple of 16 the padded indices are ridx(i0) + k (T + T/16)
    // and ridx(L - i0) - k (T + T/16)
    {
      const int i0 = c0 + tt;
      const int pa = reg::ridx(i0), pc = reg::ridx(L - i0);
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        const int i = i0 + k * T;
        if (act && i <= c1) {
          const int ia = i == L ? 0 : (T % 16 == 0 ? pa + k * (T + T / 16) : reg::ridx(i));
          const int ic = i == 0 ? 0 : (T % 16 == 0 ? pc - k * (T + T / 16) : reg::ridx(L - i));
          const float2 a = ub[ia];
          const float2 c = c_conj(ub[ic]);
          const float2 s2 = c_add(a, c), d = c_sub(a, c);
          X[i] = unpack_combine(s2, d, tw[i]);
        }
      }
    }
    flc = fln;
    rowc = rown;
  }
  cp_async_commit_wait_all();  // no copy outlives the kernel
}

// ---------------------------------------------------------------------------
// v-step with 16 values per thread (half widths L = 64 .. 1024, powers of two;
// shf_fft16.cuh): row groups of T = L/16 threads, 32/T groups per warp (two
// warps per group and a named barrier for L = 1024), eight warps per CTA,
// every lane live.  Per group, shared memory holds the FFT exchange buffer and
// the b_v stage, at a group stride that is T float2 apart modulo 16 for T < 16
// (the groups of a half-warp then use distinct banks).  The spectrum columns
// of a row are read straight from global memory (they were written by the
// preceding fan launch and sit in L2); the b_v row is staged by cp.async while
// the previous row is transformed.  The packing pairs X_n with X_{L-n} and the
// unpacking Z_i with Z_{L-i}, which lane (T - tt) mod T holds at register
// 15 - q (lane 0 holds its own partners): for T <= 32 one warp shuffle per
// value replaces a round trip through shared memory; for T = 64 the partner
// is in the other warp, and X_{L-n} is read from L2 and Z_{L-i} through the
// exchange buffer.
// ---------------------------------------------------------------------------
template <int L, int MODE = 0>
struct Row16Geo {
  static constexpr int T = L / 16;
  static constexpr int GPW = T <= 32 ? 32 / T : 0;          // groups per warp (T <= 32)
  static constexpr int NTH = 256;
  static constexpr int RPC = T <= 32 ? 8 * GPW : NTH / T;    // groups per CTA
  static constexpr int BUF = even2(reg::row_buf(L));         // exchange buffer
  static constexpr int SC = MODE == 1 ? L / 4 : 0;           // adjoint: codes of the row (2L bytes)
  static constexpr int SD = MODE == 1 ? even2(T) : 0;        // adjoint: one double per thread
  static constexpr int RAW = BUF + L + SC + SD;              // + b_v (or its adjoint) stage (L float2)
  static constexpr int STRIDE = T >= 16 ? RAW : RAW + ((T - RAW % 16) % 16 + 16) % 16;
  static constexpr int TW = even2(L + 1);                    // exp(-2 pi i m / W), m <= L
  static constexpr int PT = even2(r16::Passes<L>::TWSIZE);   // per-pass twiddles
  static constexpr int TOTAL = TW + PT + RPC * STRIDE;       // float2 per CTA
};

// MODE 0: the v-step (with optional codes); MODE 1: its adjoint, as MODE 1 of
// k_wrow_vstep (codes staged with the b_v row; each thread sums its 32
// threshold terms in FP32 in a fixed order, the group's partials are added in
// FP64 in thread order).
template <int L, int MODE>
__global__ void __launch_bounds__(256, 2)
    k_wrow_vstep16(float2* __restrict__ Y, float* __restrict__ bv, const float* __restrict__ thr,
                   const int2* __restrict__ ranges, int H, int Whp, int eta, int l0, int f0, int nf, int nv,
                   float scale, const float2* __restrict__ twW, signed char* __restrict__ code,
                   double* __restrict__ tpart) {
  using G = Row16Geo<L, MODE>;
  constexpr int T = G::T;
  constexpr int RPC = G::RPC;
  extern __shared__ __align__(16) float2 sm[];
  float2* tw = sm;
  float2* pt = tw + G::TW;
  const int lane = threadIdx.x & 31;
  const int tt = threadIdx.x & (T - 1);
  const int grp = threadIdx.x / T;
  const int partner = T <= 32 ? (lane - tt) + ((T - tt) & (T - 1)) : 0;  // shuffle source (T <= 32)
  const int bar = 1 + grp;                                               // named barrier (T = 64)
  float2* fb = pt + G::PT + grp * G::STRIDE;
  float2* sB = fb + G::BUF;
  const char2* sC = reinterpret_cast<const char2*>(sB + L);
  double* sD = reinterpret_cast<double*>(sB + L + G::SC);
  const int Gn = gridDim.x * RPC;
  const int gid = blockIdx.x * RPC + grp;
  const int rows = nv * H;
  const int niter = (rows + Gn - 1) / Gn;  // the same for every group: every lane takes part in the shuffles
  // label and filter of pair fl
  auto pair_of = [&](int fl, int& lab, int& f) {
    const int q = fl / nf;
    lab = l0 + q;
    f = f0 + fl - q * nf;
  };
  const uint64_t pol = evict_first_policy();
  const size_t W = 2 * static_cast<size_t>(L);
  const int cmask = reg::col_batch(H) - 1;
  const int gq = Gn / H, gr = Gn - gq * H;
  auto advance = [&](int& fl, int& row) {
    fl += gq;
    row += gr;
    if (row >= H) {
      row -= H;
      ++fl;
    }
  };
  auto request_b = [&](int fl, int row) {
    if (fl >= nv) return;
    int lab, f;
    pair_of(fl, lab, f);
    const size_t rix = (static_cast<size_t>(lab) * eta + f) * H + row;
    const float2* B = reinterpret_cast<const float2*>(bv) + rix * L;
#pragma unroll
    for (int q = tt; q < L / 2; q += T) cp_async16(sB + 2 * q, B + 2 * q, true, pol);
    if (MODE == 1) {  // 2L bytes of codes: L/8 = 2T chunks of 16 bytes
      const signed char* Cr = code + rix * (2 * static_cast<size_t>(L));
#pragma unroll
      for (int q = tt; q < L / 8; q += T) cp_async16(sB + L + 2 * q, Cr + 16 * q, true, pol);
    }
  };

  int flc = gid / H, rowc = gid - flc * H;
  request_b(flc, rowc);  // b_v was last written by an earlier, completed grid
  load_table(tw, twW, L + 1);
  r16::build_pass_twiddles<L, 2>(pt, twW, threadIdx.x, blockDim.x);
  pdl_wait();
  pdl_trigger();
  __syncthreads();
  for (int it = 0; it < niter; ++it) {
    const bool live = flc < nv;
    const int fl = live ? flc : 0, row = live ? rowc : 0;
    int label, f;
    pair_of(fl, label, f);
    int fln = flc, rown = rowc;
    advance(fln, rown);
    const int2 rg = ranges[f];
    const bool any = live && rg.x <= rg.y;
    const int c0 = any ? (rg.x & ~cmask) : L + 1;
    const int c1 = any ? min(L, (rg.y | cmask)) : -1;
    const float th = thr[f];
    const size_t rix = (static_cast<size_t>(label) * eta + f) * H + row;
    float2* X = Y + (static_cast<size_t>(fl) * H + row) * Whp;
    // the next row's spectrum columns into L1 (one 128-byte line per thread
    // and step), so that its loads a row from now do not wait on L2
    if (fln < nv) {
      int labn, fn;
      pair_of(fln, labn, fn);
      const int2 rgn = ranges[fn];
      if (rgn.x <= rgn.y) {
        const int n0 = rgn.x & ~cmask, n1 = min(L, (rgn.y | cmask));
        const char* base = reinterpret_cast<const char*>(Y + (static_cast<size_t>(fln) * H + rown) * Whp + n0);
        const int lines = ((n1 - n0 + 1) * 8 + 127) / 128;
        for (int ln = tt; ln < lines; ln += T) asm volatile("prefetch.global.L1 [%0];" ::"l"(base + 128 * ln));
      }
    }
    float2 v[16];
    if constexpr (T <= 32) {
      // inverse packing (r16::pack_step), X_{L-n} from the partner lane
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const int n = tt + k * T;
        v[k] = (n >= c0 && n <= c1) ? __ldca(X + n) : make_float2(0.f, 0.f);
      }
      float2 prev = (c1 >= L) ? __ldca(X + L) : make_float2(0.f, 0.f);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        float2 ra, rb;
        ra.x = __shfl_sync(0xffffffffu, v[15 - k].x, partner);
        ra.y = __shfl_sync(0xffffffffu, v[15 - k].y, partner);
        rb.x = __shfl_sync(0xffffffffu, v[k].x, partner);
        rb.y = __shfl_sync(0xffffffffu, v[k].y, partner);
        r16::pack_step<L>(v, k, tt, ra, rb, prev, tw);
      }
    } else {
      // the partner lane is in the group's other warp: X_{L-n} is read from L2 as well
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const int n = tt + k * T, m = L - n;
        const float2 a = (n >= c0 && n <= c1) ? __ldca(X + n) : make_float2(0.f, 0.f);
        const float2 c = (m >= c0 && m <= c1) ? c_conj(__ldca(X + m)) : make_float2(0.f, 0.f);
        const float2 s2 = c_add(a, c), d = c_sub(a, c);
        v[k] = pack_combine(s2, d, tw[n]);
      }
    }
    r16::row_fft<L, +1>(v, tt, fb, pt, bar);
    cp_async_commit_wait_all();  // this lane's part of the b_v row
    r16::group_sync<L>(bar);     // ... and the group's
    if (live) {
      float2* b2 = reinterpret_cast<float2*>(bv) + rix * L;
      if constexpr (MODE == 0) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const float2 g = c_fma2(make_float2(scale, scale), v[k], sB[tt + k * T]);
          const float2 c = make_float2(fminf(fmaxf(g.x, -th), th), fminf(fmaxf(g.y, -th), th));
          __stcs(b2 + tt + k * T, c);
          if (code)
            reinterpret_cast<char2*>(code + rix * W)[tt + k * T] = make_char2(clip_code(g.x, th), clip_code(g.y, th));
          v[k] = c_fma2(make_float2(-2.f, -2.f), c, g);  // g - 2 clip(g)
        }
      } else {
        float tacc = 0.f;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const float2 bo = sB[tt + k * T];
          const char2 m = sC[tt + k * T];
          const float dx = scale * v[k].x, dy = scale * v[k].y;
          const float nx = m.x == 0 ? bo.x - dx : dx;
          const float ny = m.y == 0 ? bo.y - dy : dy;
          tacc = fmaf(static_cast<float>(m.x), fmaf(-2.f, dx, bo.x), tacc);
          tacc = fmaf(static_cast<float>(m.y), fmaf(-2.f, dy, bo.y), tacc);
          __stcs(b2 + tt + k * T, make_float2(nx, ny));
          v[k] = make_float2(nx, ny);
        }
        sD[tt] = static_cast<double>(tacc);
      }
    } else {
#pragma unroll
      for (int k = 0; k < 16; ++k) v[k] = make_float2(0.f, 0.f);
    }
    r16::group_sync<L>(bar);  // the b_v stage is read: refill it with the group's next row
    if (MODE == 1 && live && tt == 0) {  // the row's threshold sum, in thread order
      double sum = 0.0;
      for (int j = 0; j < T; ++j) sum += sD[j];
      tpart[rix] = sum;
    }
    request_b(fln, rown);
    r16::row_fft<L, -1>(v, tt, fb, pt, bar);
    if constexpr (T <= 32) {
      // forward unpacking (r16::unpack_value), Z_{L-i} from the partner lane
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        float2 r;
        r.x = __shfl_sync(0xffffffffu, v[15 - q].x, partner);
        r.y = __shfl_sync(0xffffffffu, v[15 - q].y, partner);
        const int i = tt + q * T;
        if (i >= c0 && i <= c1) X[i] = r16::unpack_value<L>(v, q, tt, r, tw);
      }
    } else {
      // Z_{L-i} through the exchange buffer (natural order at ridx)
      r16::group_sync<L>(bar);  // the last pass may still read the buffer
#pragma unroll
      for (int q = 0; q < 16; ++q) fb[reg::ridx(tt + q * T)] = v[q];
      r16::group_sync<L>(bar);
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int i = tt + q * T;
        if (i >= c0 && i <= c1) X[i] = r16::unpack_value<L>(v, q, tt, fb[reg::ridx((L - i) & (L - 1))], tw);
      }
    }
    if (tt == 0 && c1 >= L) X[L] = make_float2(v[0].x - v[0].y, 0.f);  // i = L: e^{-i pi} = -1
    flc = fln;
    rowc = rown;
  }
  cp_async_commit_wait_all();  // no copy outlives the kernel
}

// ---------------------------------------------------------------------------
// v-step on pairs of rows (half widths L = 64, 128): rows r and r + 1 of
// the same (label, filter) are one complex row z = a + i b of length W = 2L
// (r16::pair_pack / pair_unpack), transformed by a group of T = W/16 <= 32
// threads.  Against one half-length transform per row this drops the packing
// twiddles and the packing shuffles, and half of the exchanges.
// The b_v rows of a pair are contiguous (2W floats), staged by cp.async.
// Forward mode only (optional codes); the adjoint keeps k_wrow_vstep16.
// ---------------------------------------------------------------------------
template <int L>
struct PairGeo {
  static constexpr int W = 2 * L;
  static constexpr int T = W / 16;                           // threads per pair
  static_assert(T <= 32, "pair groups inside one warp");
  static constexpr int GPW = 32 / T;
  static constexpr int NTH = 256;
  static constexpr int RPC = 8 * GPW;                        // pair groups per CTA
  static constexpr int BUF = even2(reg::row_buf(W));         // exchange buffer (length W)
  static constexpr int RAW = BUF + W;                        // + the two b_v rows (W float2)
  static constexpr int STRIDE = T >= 16 ? RAW : RAW + ((T - RAW % 16) % 16 + 16) % 16;
  static constexpr int PT = even2(r16::Passes<W>::TWSIZE);  // per-pass twiddles (length W)
  static constexpr int TOTAL = PT + RPC * STRIDE;            // float2 per CTA
};

template <int L>
__global__ void __launch_bounds__(256, 2)
    k_wrow_vstep2r(float2* __restrict__ Y, float* __restrict__ bv, const float* __restrict__ thr,
                   const int2* __restrict__ ranges, int H, int Whp, int eta, int l0, int f0, int nf, int nv,
                   float scale, const float2* __restrict__ twW, signed char* __restrict__ code) {
  using G = PairGeo<L>;
  constexpr int T = G::T, W = G::W;
  extern __shared__ __align__(16) float2 sm[];
  float2* pt = sm;
  const int lane = threadIdx.x & 31;
  const int tt = lane & (T - 1);
  const int grp = threadIdx.x / T;
  const int partner = (lane - tt) + ((T - tt) & (T - 1));
  float2* fb = pt + G::PT + grp * G::STRIDE;
  float* sB = reinterpret_cast<float*>(fb + G::BUF);  // b_v rows r, r + 1: 2W floats
  const int Hp = H / 2;                               // row pairs per (label, filter)
  const int Gn = gridDim.x * G::RPC;
  const int gid = blockIdx.x * G::RPC + grp;
  const int pairs = nv * Hp;
  const int niter = (pairs + Gn - 1) / Gn;  // the same for every group: every lane takes part in the shuffles
  auto pair_of = [&](int fl, int& lab, int& f) {
    const int q = fl / nf;
    lab = l0 + q;
    f = f0 + fl - q * nf;
  };
  const uint64_t pol = evict_first_policy();
  const int cmask = reg::col_batch(H) - 1;
  const int gq = Gn / Hp, gr = Gn - gq * Hp;
  auto advance = [&](int& fl, int& pr) {
    fl += gq;
    pr += gr;
    if (pr >= Hp) {
      pr -= Hp;
      ++fl;
    }
  };
  auto request_b = [&](int fl, int pr) {
    if (fl >= nv) return;
    int lab, f;
    pair_of(fl, lab, f);
    const size_t rix = (static_cast<size_t>(lab) * eta + f) * H + 2 * pr;
    const float* B = bv + rix * W;
#pragma unroll
    for (int q = tt; q < W / 2; q += T) cp_async16(sB + 4 * q, B + 4 * q, true, pol);
  };

  int flc = gid / Hp, prc = gid - flc * Hp;
  request_b(flc, prc);  // b_v was last written by an earlier, completed grid
  r16::build_pass_twiddles<W, 1>(pt, twW, threadIdx.x, blockDim.x);
  pdl_wait();
  pdl_trigger();
  __syncthreads();
  for (int it = 0; it < niter; ++it) {
    const bool live = flc < nv;
    const int fl = live ? flc : 0, pr = live ? prc : 0;
    int label, f;
    pair_of(fl, label, f);
    int fln = flc, prn = prc;
    advance(fln, prn);
    const int2 rg = ranges[f];
    const bool any = live && rg.x <= rg.y;
    const int c0 = any ? (rg.x & ~cmask) : L + 1;
    const int c1 = any ? min(L, (rg.y | cmask)) : -1;
    const float th = thr[f];
    const size_t rix = (static_cast<size_t>(label) * eta + f) * H + 2 * pr;  // row a; row b = rix + 1
    float2* Xa = Y + (static_cast<size_t>(fl) * H + 2 * pr) * Whp;
    float2* Xb = Xa + Whp;
    // Z[n] = Xa[n] + i Xb[n] (n <= L), conj Xa[W-n] + i conj Xb[W-n] (n > L)
    float2 v[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int n = tt + k * T;
      const bool up = n > L;
      const int m = up ? W - n : n;
      const bool in = m >= c0 && m <= c1;
      const float2 xa = in ? __ldcg(Xa + m) : make_float2(0.f, 0.f);
      const float2 xb = in ? __ldcg(Xb + m) : make_float2(0.f, 0.f);
      v[k] = r16::pair_pack(xa, xb, up);
    }
    r16::row_fft<W, +1>(v, tt, fb, pt, 0);
    cp_async_commit_wait_all();  // this lane's part of the b_v rows
    __syncwarp();                // ... and the group's
    if (live) {
      float* b2 = bv + rix * W;
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const int m = tt + k * T;
        const float2 g = c_fma2(make_float2(scale, scale), v[k], make_float2(sB[m], sB[W + m]));  // rows a, b
        const float2 c = make_float2(fminf(fmaxf(g.x, -th), th), fminf(fmaxf(g.y, -th), th));
        __stcs(b2 + m, c.x);
        __stcs(b2 + W + m, c.y);
        if (code) {
          code[rix * W + m] = clip_code(g.x, th);
          code[(rix + 1) * W + m] = clip_code(g.y, th);
        }
        v[k] = c_fma2(make_float2(-2.f, -2.f), c, g);  // g - 2 clip(g)
      }
    } else {
#pragma unroll
      for (int k = 0; k < 16; ++k) v[k] = make_float2(0.f, 0.f);
    }
    __syncwarp();  // the b_v stage is read: refill it with the group's next pair
    request_b(fln, prn);
    r16::row_fft<W, -1>(v, tt, fb, pt, 0);
    // Xa[k], Xb[k] for k = tt + q T <= L from D_k (register q) and D_{W-k}
#pragma unroll
    for (int q = 0; q <= 8; ++q) {
      float2 r;
      r.x = __shfl_sync(0xffffffffu, v[15 - q].x, partner);
      r.y = __shfl_sync(0xffffffffu, v[15 - q].y, partner);
      const int k = tt + q * T;
      if (k >= c0 && k <= c1) {
        float2 xa, xb;
        r16::pair_unpack(v[q], r16::pair_partner(tt, r, v[(16 - q) & 15]), xa, xb);
        Xa[k] = xa;
        Xb[k] = xb;
      }
    }
    flc = fln;
    prc = prn;
  }
  cp_async_commit_wait_all();  // no copy outlives the kernel
}

// ---------------------------------------------------------------------------
// v-step with V values per thread for the half widths with an odd factor
// (L = 12 T or 20 T, T = 2..32) and for L = 1024 (V = T = 32; shf_fftv.cuh):
// row groups of T threads, 32/T groups per warp, eight warps per CTA (twelve
// for V = 32), every lane live; the layout, the b_v stage, the L1 prefetch of
// the next row's spectrum columns and the partner-lane packing are those of
// k_wrow_vstep16 for T <= 32.  Forward mode (optional codes); the adjoint
// keeps k_wrow_vstep16 / k_wrow_vstep.
// ---------------------------------------------------------------------------
template <int L>
struct RowVGeo {
  static constexpr int V = rv::vals_for(L);
  static constexpr int T = L / V;
  static constexpr int GPW = 32 / T;                           // groups per warp
  // 32 values per thread: 17 KB of buffers per row, 12 one-warp rows in one
  // CTA per SM (219 KB) with up to 168 registers per thread
  static constexpr int NTH = V == 32 ? 384 : 256;
  static constexpr int MINB = V == 32 ? 1 : 2;
  static constexpr int RPC = NTH / 32 * GPW;                   // groups per CTA
  static constexpr int BUF = even2(rv::row_buf(L));            // exchange buffer
  static constexpr int RAW = BUF + L;                          // + the b_v stage (L float2)
  static constexpr int STRIDE = T >= 16 ? RAW : RAW + ((T - RAW % 16) % 16 + 16) % 16;
  static constexpr int TW = even2(L + 1);                      // exp(-2 pi i m / W), m <= L
  static constexpr int PT = even2(rv::Passes<L>::TWSIZE);      // per-pass twiddles
  static constexpr int TOTAL = TW + PT + RPC * STRIDE;         // float2 per CTA
};

template <int L>
__global__ void __launch_bounds__(RowVGeo<L>::NTH, RowVGeo<L>::MINB)
    k_wrow_vstepv(float2* __restrict__ Y, float* __restrict__ bv, const float* __restrict__ thr,
                  const int2* __restrict__ ranges, int H, int Whp, int eta, int l0, int f0, int nf, int nv,
                  float scale, const float2* __restrict__ twW, signed char* __restrict__ code) {
  using G = RowVGeo<L>;
  constexpr int T = G::T, V = G::V, RPC = G::RPC;
  extern __shared__ __align__(16) float2 sm[];
  float2* tw = sm;
  float2* pt = tw + G::TW;
  const int lane = threadIdx.x & 31;
  const int tt = threadIdx.x & (T - 1);
  const int grp = threadIdx.x / T;
  const int partner = (lane - tt) + ((T - tt) & (T - 1));  // shuffle source
  float2* fb = pt + G::PT + grp * G::STRIDE;
  float2* sB = fb + G::BUF;
  const int Gn = gridDim.x * RPC;
  const int gid = blockIdx.x * RPC + grp;
  const int rows = nv * H;
  const int niter = (rows + Gn - 1) / Gn;  // the same for every group: every lane takes part in the shuffles
  auto pair_of = [&](int fl, int& lab, int& f) {
    const int q = fl / nf;
    lab = l0 + q;
    f = f0 + fl - q * nf;
  };
  const uint64_t pol = evict_first_policy();
  const size_t W = 2 * static_cast<size_t>(L);
  const int cmask = reg::col_batch(H) - 1;
  const int gq = Gn / H, gr = Gn - gq * H;
  auto advance = [&](int& fl, int& row) {
    fl += gq;
    row += gr;
    if (row >= H) {
      row -= H;
      ++fl;
    }
  };
  auto request_b = [&](int fl, int row) {
    if (fl >= nv) return;
    int lab, f;
    pair_of(fl, lab, f);
    const size_t rix = (static_cast<size_t>(lab) * eta + f) * H + row;
    const float2* B = reinterpret_cast<const float2*>(bv) + rix * L;
#pragma unroll
    for (int q = tt; q < L / 2; q += T) cp_async16(sB + 2 * q, B + 2 * q, true, pol);
  };

  int flc = gid / H, rowc = gid - flc * H;
  request_b(flc, rowc);  // b_v was last written by an earlier, completed grid
  load_table(tw, twW, L + 1);
  rv::build_pass_twiddles<L, 2>(pt, twW, threadIdx.x, blockDim.x);
  pdl_wait();
  pdl_trigger();
  __syncthreads();
  for (int it = 0; it < niter; ++it) {
    const bool live = flc < nv;
    const int fl = live ? flc : 0, row = live ? rowc : 0;
    int label, f;
    pair_of(fl, label, f);
    int fln = flc, rown = rowc;
    advance(fln, rown);
    const int2 rg = ranges[f];
    const bool any = live && rg.x <= rg.y;
    const int c0 = any ? (rg.x & ~cmask) : L + 1;
    const int c1 = any ? min(L, (rg.y | cmask)) : -1;
    const float th = thr[f];
    const size_t rix = (static_cast<size_t>(label) * eta + f) * H + row;
    float2* X = Y + (static_cast<size_t>(fl) * H + row) * Whp;
    // the next row's spectrum columns into L1 (one 128-byte line per thread and step)
    if (fln < nv) {
      int labn, fn;
      pair_of(fln, labn, fn);
      const int2 rgn = ranges[fn];
      if (rgn.x <= rgn.y) {
        const int n0 = rgn.x & ~cmask, n1 = min(L, (rgn.y | cmask));
        const char* base = reinterpret_cast<const char*>(Y + (static_cast<size_t>(fln) * H + rown) * Whp + n0);
        const int lines = ((n1 - n0 + 1) * 8 + 127) / 128;
        for (int ln = tt; ln < lines; ln += T) asm volatile("prefetch.global.L1 [%0];" ::"l"(base + 128 * ln));
      }
    }
    // inverse packing (rv::pack_step), X_{L-n} from the partner lane
    float2 v[V];
#pragma unroll
    for (int k = 0; k < V; ++k) {
      const int n = tt + k * T;
      v[k] = (n >= c0 && n <= c1) ? __ldca(X + n) : make_float2(0.f, 0.f);
    }
    float2 prev = (c1 >= L) ? __ldca(X + L) : make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < V / 2; ++k) {
      float2 ra, rb;
      ra.x = __shfl_sync(0xffffffffu, v[V - 1 - k].x, partner);
      ra.y = __shfl_sync(0xffffffffu, v[V - 1 - k].y, partner);
      rb.x = __shfl_sync(0xffffffffu, v[k].x, partner);
      rb.y = __shfl_sync(0xffffffffu, v[k].y, partner);
      rv::pack_step<L>(v, k, tt, ra, rb, prev, tw);
    }
    rv::row_fft<L, +1>(v, tt, fb, pt);
    cp_async_commit_wait_all();  // this lane's part of the b_v row
    __syncwarp();                // ... and the group's
    if (live) {
      float2* b2 = reinterpret_cast<float2*>(bv) + rix * L;
#pragma unroll
      for (int k = 0; k < V; ++k) {
        const float2 g = c_fma2(make_float2(scale, scale), v[k], sB[tt + k * T]);
        const float2 c = make_float2(fminf(fmaxf(g.x, -th), th), fminf(fmaxf(g.y, -th), th));
        __stcs(b2 + tt + k * T, c);
        if (code)
          reinterpret_cast<char2*>(code + rix * W)[tt + k * T] = make_char2(clip_code(g.x, th), clip_code(g.y, th));
        v[k] = c_fma2(make_float2(-2.f, -2.f), c, g);  // g - 2 clip(g)
      }
    } else {
#pragma unroll
      for (int k = 0; k < V; ++k) v[k] = make_float2(0.f, 0.f);
    }
    __syncwarp();  // the b_v stage is read: refill it with the group's next row
    request_b(fln, rown);
    rv::row_fft<L, -1>(v, tt, fb, pt);
    // forward unpacking (rv::unpack_value), Z_{L-i} from the partner lane
#pragma unroll
    for (int q = 0; q < V; ++q) {
      float2 r;
      r.x = __shfl_sync(0xffffffffu, v[V - 1 - q].x, partner);
      r.y = __shfl_sync(0xffffffffu, v[V - 1 - q].y, partner);
      const int i = tt + q * T;
      if (i >= c0 && i <= c1) X[i] = rv::unpack_value<L>(v, q, tt, r, tw);
    }
    if (tt == 0 && c1 >= L) X[L] = make_float2(v[0].x - v[0].y, 0.f);  // i = L: e^{-i pi} = -1
    flc = fln;
    rowc = rown;
  }
  cp_async_commit_wait_all();  // no copy outlives the kernel
}

// Geometry of the u/w-step kernel: a CTA takes NR rows and runs one row
// group per (row, label) — K NR groups, laid out like RowGeo's groups (32/T
// per warp, T/32 warps each, or packed back to back; group slots past K NR
// idle).
template <int L>
struct UstepGeo {
  using RG = RowGeo<L>;
  static constexpr int T = RG::T;
  __host__ __device__ static int rows(int K) {
    const int nr = !RG::TILE ? (256 / T) / K : (T <= 32 ? (8 * RG::GPW) / K : 8 / (RG::WPG * K));
    return nr < 1 ? 1 : nr;
  }
  __host__ __device__ static int groups(int K) { return K * rows(K); }
  // threads of the CTA, and the group slots they hold
  __host__ __device__ static int warps(int K) {
    return !RG::TILE ? (groups(K) * T + 31) / 32
                     : (T <= 32 ? (groups(K) + RG::GPW - 1) / RG::GPW : groups(K) * RG::WPG);
  }
  __host__ __device__ static int slots(int K) {
    return !RG::TILE ? (32 * warps(K) + T - 1) / T : (T <= 32 ? warps(K) * RG::GPW : groups(K));
  }
  // the largest CTA over K <= 8, and the CTAs per SM to ask the compiler for
  static constexpr int MAXTH = !RG::TILE ? (8 * T > 256 ? (8 * T + 31) / 32 * 32 : 256)
                                         : (T <= 32 ? 256 : 256 * RG::WPG);
  static constexpr int MINB = MAXTH <= 256 ? 2 : 1;  // room for the phase-2 operand prefetch
};

// u-step (u = 1/2 [S^T(v - b_v) + (w - b_w) - gamma s], A^T A = 2I), w-step
// (pixelwise simplex projection of g_w = b_w + u), b_w = g_w - w, and the row
// spectra of u for the next analysis (Sec. 3).  Phase 1: group (r, k) inverts
// the spectrum row of label k into U[k][r]; phase 2: all threads do the
// pointwise steps over the CTA's pixels and labels; phase 3: group (r, k)
// transforms U[k][r] (now u) forward into Ur.
template <int L, int KMAX>
__global__ void __launch_bounds__(UstepGeo<L>::MAXTH, UstepGeo<L>::MINB) k_wrow_ustep(const float2* __restrict__ Tsp, const float* __restrict__ s,
                                                     float* __restrict__ w, float* __restrict__ bw,
                                                     float* __restrict__ u, float2* __restrict__ Ur, int K, int H,
                                                     float scale, float gamma, const float2* __restrict__ twW) {
  using UG = UstepGeo<L>;
  constexpr int T = L / 8;
  constexpr int BUF = reg::row_buf(L);
  constexpr int NBUF = T <= 32 ? 1 : 2;
  constexpr int Wh = L + 1;
  const int NR = UG::rows(K), NG = K * NR;
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* pt = tw + (L + 1);
  int grp, tt;
  bool act;
  RowGeo<L>::locate(grp, tt, act);
  float2* b0 = pt + reg::Passes<L>::TWSIZE + grp * NBUF * BUF;
  float2* b1 = b0 + (NBUF - 1) * BUF;
  float2* U = pt + reg::Passes<L>::TWSIZE + UG::slots(K) * NBUF * BUF;  // [k][r][L]
  const bool real = grp < NG;  // groups past K NR only take part in barriers
  const int r = real ? grp / K : 0, k = real ? grp - (grp / K) * K : 0;
  const int bar = 1 + grp;
  const int row = blockIdx.x * NR + r;
  const bool live = real && row < H;
  const int rowc = row < H ? row : 0;
  const size_t HL = static_cast<size_t>(H) * L, HWh = static_cast<size_t>(H) * Wh;
  float2* Uk = U + (static_cast<size_t>(k) * NR + r) * L;
  load_table(tw, twW, L + 1);
  reg::build_pass_twiddles<L, 2>(pt, twW, threadIdx.x, blockDim.x);
  pdl_wait();
  pdl_trigger();
  // the operands of this thread's first PRE phase-2 items (w, b_w, s: written
  // by earlier, completed grids) are requested now, so that their latency
  // overlaps phase 1
  // (K <= 4 only: with K up to 8 the registers cost more than the overlap gains,
  // 424 -> 451 us per 2048^2 iteration)
  constexpr int PRE = KMAX <= 4 ? 2 : 0;
  constexpr int PREA = PRE > 0 ? PRE : 1;
  const float2* s2 = reinterpret_cast<const float2*>(s);
  float2* w2 = reinterpret_cast<float2*>(w);
  float2* bw2 = reinterpret_cast<float2*>(bw);
  float2* u2 = reinterpret_cast<float2*>(u);
  float2 pw[PREA][KMAX], pb[PREA][KMAX], ps[PREA][KMAX];
#pragma unroll
  for (int j = 0; j < PRE; ++j) {
    const int i = threadIdx.x + j * blockDim.x;
    const int ri = i / L, n = i - ri * L;
    const int prow = blockIdx.x * NR + ri;
    const bool ok = i < NR * L && prow < H;
    const size_t pix = static_cast<size_t>(ok ? prow : 0) * L + n;
#pragma unroll
    for (int q = 0; q < KMAX; ++q) {
      const bool lq = ok && q < K;
      pw[j][q] = lq ? w2[HL * q + pix] : make_float2(0.f, 0.f);
      pb[j][q] = lq ? bw2[HL * q + pix] : make_float2(0.f, 0.f);
      ps[j][q] = lq ? s2[HL * q + pix] : make_float2(0.f, 0.f);
    }
  }
  __syncthreads();
  // phase 1: S^T(v - b_v) on row r of label k
  {
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
    if (NBUF == 1)
      reg::row_fft1<L, +1>(v, tt, b0, pt, bar);
    else
      reg::row_fft<L, +1>(v, tt, b0, b1, pt, bar);
    if (real && act) {
#pragma unroll
      for (int e = 0; e < 8; ++e) Uk[tt + e * T] = c_scale(v[e], scale);
    }
  }
  __syncthreads();
  // phase 2: pointwise u-step, projection and b_w update (two pixels per item)
  {
    const float hg = 0.5f * gamma;
    // one item: `get(q, pix, wv, bv, sv)` supplies label q's w, b_w and s
    auto item = [&](int i, auto get) {
      const int ri = i / L, n = i - ri * L;
      const int prow = blockIdx.x * NR + ri;
      if (prow >= H) return;
      const size_t pix = static_cast<size_t>(prow) * L + n;
      float gx[KMAX], gy[KMAX];
#pragma unroll
      for (int q = 0; q < KMAX; ++q) {
        gx[q] = 0.f;
        gy[q] = 0.f;
        if (q < K) {
          float2 wv, bv, sv;
          get(q, pix, wv, bv, sv);
          float2* Uq = U + (static_cast<size_t>(q) * NR + ri) * L + n;
          const float2 st = *Uq;
          const float ux = 0.5f * (st.x + (wv.x - bv.x)) - hg * sv.x;
          const float uy = 0.5f * (st.y + (wv.y - bv.y)) - hg * sv.y;
          u2[HL * q + pix] = make_float2(ux, uy);
          *Uq = make_float2(ux, uy);
          gx[q] = bv.x + ux;
          gy[q] = bv.y + uy;
        }
      }
      float px[KMAX], py[KMAX];
#pragma unroll
      for (int q = 0; q < KMAX; ++q) {
        px[q] = gx[q];
        py[q] = gy[q];
      }
      simplex_project<KMAX>(px, K);
      simplex_project<KMAX>(py, K);
#pragma unroll
      for (int q = 0; q < KMAX; ++q)
        if (q < K) {
          w2[HL * q + pix] = make_float2(px[q], py[q]);
          bw2[HL * q + pix] = make_float2(gx[q] - px[q], gy[q] - py[q]);
        }
    };
#pragma unroll
    for (int j = 0; j < PRE; ++j) {
      const int i = threadIdx.x + j * blockDim.x;
      if (i < NR * L)
        item(i, [&](int q, size_t, float2& wv, float2& bv, float2& sv) {
          wv = pw[j][q];
          bv = pb[j][q];
          sv = ps[j][q];
        });
    }
    for (int i = threadIdx.x + PRE * blockDim.x; i < NR * L; i += blockDim.x)
      item(i, [&](int q, size_t pix, float2& wv, float2& bv, float2& sv) {
        wv = w2[HL * q + pix];
        bv = bw2[HL * q + pix];
        sv = s2[HL * q + pix];
      });
  }
  __syncthreads();
  // phase 3: row spectrum of u on row r of label k
  {
    float2 v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = Uk[tt + e * T];
    if (NBUF == 1)
      reg::row_fft1<L, -1>(v, tt, b0, pt, bar);
    else
      reg::row_fft<L, -1>(v, tt, b0, b1, pt, bar);
    float2* ub = NBUF == 1 ? b0 : b1;
    reg::group_sync<T>(bar);
#pragma unroll
    for (int e = 0; e < 8; ++e) ub[reg::ridx(tt + e * T)] = v[e];
    reg::group_sync<T>(bar);
    if (live && act) {
      float2* X = Ur + HWh * k + static_cast<size_t>(row) * Wh;
      for (int i = tt; i <= L; i += T) {
        const float2 a = ub[reg::ridx(i == L ? 0 : i)];
        const float2 c = c_conj(ub[reg::ridx(i == 0 ? 0 : L - i)]);
        const float2 sm2 = c_add(a, c), d = c_sub(a, c);
        const float2 t = c_mul(tw[i], d);
        X[i] = make_float2(0.5f * (sm2.x + t.y), 0.5f * (sm2.y - t.x));
      }
    }
  }
}

}  // namespace

namespace {

template <int L, int MODE>
size_t vstep_smem() {
  return sizeof(float2) * RowGroupSmem<L, MODE>::TOTAL;
}

template <int L>
size_t ustep_smem(int K) {
  using UG = UstepGeo<L>;
  const int nbuf = L / 8 <= 32 ? 1 : 2;
  return sizeof(float2) * ((L + 1) + reg::Passes<L>::TWSIZE + static_cast<size_t>(UG::slots(K)) * nbuf * reg::row_buf(L) +
                           static_cast<size_t>(K) * UG::rows(K) * L);
}

// Half widths served by the radix-16 v-step and its adjoint.
__host__ __device__ constexpr bool use_r16(int L) { return L == 64 || L == 128 || L == 256 || L == 512 || L == 1024; }
// the radix-16 instance of a dispatch case (a valid placeholder where not used)
__host__ __device__ constexpr int r16_len(int L) { return use_r16(L) ? L : 64; }

template <int L, int MODE>
size_t vstep16_smem() {
  return sizeof(float2) * Row16Geo<r16_len(L), MODE>::TOTAL;
}

// Half widths whose forward v-step runs on pairs of rows: 64 and 128, where a
// pair takes one exchange where two single rows take two (measured: the
// unrolled 256^2 sweeps 1695 -> 1745 Mpixel*label*iter/s).  At 256 a pair
// needs three passes where a row needs two, and the one-row kernel is faster
// (v-step 156 against 164 us per 512^2 iteration).
__host__ __device__ constexpr bool use_pair(int L) { return L == 64 || L == 128; }
__host__ __device__ constexpr int pair_len(int L) { return use_pair(L) ? L : 64; }
template <int L>
size_t pair_smem() {
  return sizeof(float2) * PairGeo<pair_len(L)>::TOTAL;
}

// Half widths whose forward v-step can run on V values per thread
// (shf_fftv.cuh): 12 T or 20 T with T = 2..32.
__host__ __device__ constexpr bool use_v(int L) { return rv::supported(L); }
__host__ __device__ constexpr int v_len(int L) { return use_v(L) ? L : 24; }
template <int L>
size_t vstepv_smem() {
  return sizeof(float2) * RowVGeo<v_len(L)>::TOTAL;
}

template <int L>
cudaError_t prepare_row_t() {
  cudaError_t e = allow_smem(k_wrow_vstep<L, 0>, vstep_smem<L, 0>());
  if (e == cudaSuccess) e = allow_smem(k_wrow_vstep<L, 1>, vstep_smem<L, 1>());
  if constexpr (use_r16(L)) {
    if (e == cudaSuccess) e = allow_smem(k_wrow_vstep16<L, 0>, vstep16_smem<L, 0>());
    if (e == cudaSuccess) e = allow_smem(k_wrow_vstep16<L, 1>, vstep16_smem<L, 1>());
  }
  if constexpr (use_pair(L))
    if (e == cudaSuccess) e = allow_smem(k_wrow_vstep2r<L>, pair_smem<L>());
  if constexpr (use_v(L))
    if (e == cudaSuccess) e = allow_smem(k_wrow_vstepv<L>, vstepv_smem<L>());
  // the u/w-step's shared memory depends on K (rows per CTA): the largest over
  // the K each instance serves (2..4 and 5..8)
  size_t m4 = 0, m8 = 0;
  for (int K = 2; K <= 8; ++K) (K <= 4 ? m4 : m8) = std::max(K <= 4 ? m4 : m8, ustep_smem<L>(K));
  if (e == cudaSuccess) e = allow_smem(k_wrow_ustep<L, 4>, m4);
  if (e == cudaSuccess) e = allow_smem(k_wrow_ustep<L, 8>, m8);
  return e;
}

template <int L>
cudaError_t ustep_t(const Geo& g, const float2* T, const float* s, float* w, float* bw, float* u, float2* Ur, int K,
                    float gamma, float scale, cudaStream_t st) {
  using UG = UstepGeo<L>;
  const int nr = UG::rows(K);
  const dim3 grid((g.H + nr - 1) / nr), block(32 * UG::warps(K));
  if (K <= 4)
    return launch_pdl(k_wrow_ustep<L, 4>, grid, block, ustep_smem<L>(K), st, T, s, w, bw, u, Ur, K, g.H, scale,
                      gamma, g.twW);
  return launch_pdl(k_wrow_ustep<L, 8>, grid, block, ustep_smem<L>(K), st, T, s, w, bw, u, Ur, K, g.H, scale,
                    gamma, g.twW);
}

}  // namespace

cudaError_t prepare_row_kernels() {
#define SHF_PREP(N) \
  if (e == cudaSuccess) e = prepare_row_t<N>();
  cudaError_t e = cudaSuccess;
  SHF_FAST_SIZES(SHF_PREP)
#undef SHF_PREP
  return e;
}

// The forward v-step a plan's variant selects at half width L (the default:
// pairs of rows at 64 and 128, radix-16 rows at the other powers of two up to
// 1024, 8 values per thread elsewhere).
int row_variant(int L, int mode, int variant) {
  if (mode == 1) return use_r16(L) ? kRow16 : kRow8;
  if (variant == kRowDefault) return use_pair(L) ? kRowPair : (use_r16(L) ? kRow16 : (use_v(L) ? kRowV : kRow8));
  if (variant == kRowPair && !use_pair(L)) return kRow8;
  if (variant == kRow16 && !use_r16(L)) return kRow8;
  if (variant == kRowV && !use_v(L)) return kRow8;
  return variant;
}

bool row_kernel_ok(int L, int variant) {
  return variant == kRowDefault || variant == kRow8 || (variant == kRow16 && use_r16(L)) ||
         (variant == kRowPair && use_pair(L)) || (variant == kRowV && use_v(L));
}

int row_ctas_per_sm(int L, int mode, int variant) {
  int fit = 0;
  cudaError_t e = cudaErrorInvalidValue;
  const int v = row_variant(L, mode, variant);
  switch (L) {
#define SHF_OCC(N)                                                                                              \
  case N:                                                                                                       \
    if (v == kRowPair)                                                                                          \
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, k_wrow_vstep2r<pair_len(N)>, 256, pair_smem<N>());  \
    else if (v == kRowV)                                                                                        \
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, k_wrow_vstepv<v_len(N)>, RowVGeo<v_len(N)>::NTH,   \
                                                        vstepv_smem<N>());                                      \
    else if (v == kRow16)                                                                                       \
      e = mode == 0 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, k_wrow_vstep16<r16_len(N), 0>, 256,   \
                                                                    vstep16_smem<N, 0>())                       \
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, k_wrow_vstep16<r16_len(N), 1>, 256,   \
                                                                    vstep16_smem<N, 1>());                      \
    else                                                                                                        \
      e = mode == 0 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, k_wrow_vstep<N, 0>, RowGeo<N>::NTH,   \
                                                                    vstep_smem<N, 0>())                         \
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, k_wrow_vstep<N, 1>, RowGeo<N>::NTH,   \
                                                                    vstep_smem<N, 1>());                        \
    break;
    SHF_FAST_SIZES(SHF_OCC)
#undef SHF_OCC
    default: break;
  }
  return e == cudaSuccess ? fit : 0;
}

int row_groups_per_cta(int L, int mode, int variant) {
  const int v = row_variant(L, mode, variant);
  switch (L) {
#define SHF_CASE(N)                                        \
  case N:                                                  \
    if (v == kRowPair) return 2 * PairGeo<pair_len(N)>::RPC; /* rows */ \
    if (v == kRowV) return RowVGeo<v_len(N)>::RPC;                        \
    return v == kRow16 ? Row16Geo<r16_len(N)>::RPC : RowGeo<N>::RPC;
    SHF_FAST_SIZES(SHF_CASE)
#undef SHF_CASE
    default: return 0;
  }
}

cudaError_t row_shrink(const Geo& g, int ctas, float2* Y, float* bv, const float* thr, int Whp, const Wave& wv,
                       float scale, signed char* code, int variant, cudaStream_t st) {
  const int v = row_variant(g.L, 0, variant);
  switch (g.L) {
#define SHF_CASE(N)                                                                                                \
  case N:                                                                                                          \
    if (v == kRowPair)                                                                                             \
      return launch_pdl(k_wrow_vstep2r<pair_len(N)>, dim3(ctas), dim3(256), pair_smem<N>(), st, Y, bv, thr,      \
                        g.ranges, g.H, Whp, g.eta, wv.l0, wv.f0, wv.nf, wv.nv, scale, g.twW, code);              \
    if (v == kRowV)                                                                                                \
      return launch_pdl(k_wrow_vstepv<v_len(N)>, dim3(ctas), dim3(RowVGeo<v_len(N)>::NTH), vstepv_smem<N>(), st,  \
                        Y, bv, thr,                                                                              \
                        g.ranges, g.H, Whp, g.eta, wv.l0, wv.f0, wv.nf, wv.nv, scale, g.twW, code);              \
    if (v == kRow16)                                                                                               \
      return launch_pdl(k_wrow_vstep16<r16_len(N), 0>, dim3(ctas), dim3(256), vstep16_smem<N, 0>(), st, Y, bv,    \
                        thr, g.ranges, g.H, Whp, g.eta, wv.l0, wv.f0, wv.nf, wv.nv, scale, g.twW, code,            \
                        static_cast<double*>(nullptr));                                                            \
    return launch_pdl(k_wrow_vstep<N, 0>, dim3(ctas), dim3(RowGeo<N>::NTH), vstep_smem<N, 0>(), st, Y, bv, thr,   \
                      g.ranges, g.H, Whp, g.eta, wv.l0, wv.f0, wv.nf, wv.nv, scale, g.twW, code,                    \
                      static_cast<double*>(nullptr));
    SHF_FAST_SIZES(SHF_CASE)
#undef SHF_CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t row_adjoint(const Geo& g, int ctas, float2* Y, float* bvbar, const float* thr, int Whp, const Wave& wv,
                        float scale, const signed char* code, double* tpart, cudaStream_t st) {
  switch (g.L) {
#define SHF_CASE(N)                                                                                                  \
  case N:                                                                                                            \
    if (use_r16(N))                                                                                                  \
      return launch_pdl(k_wrow_vstep16<r16_len(N), 1>, dim3(ctas), dim3(256), vstep16_smem<N, 1>(), st, Y, bvbar,   \
                        thr, g.ranges, g.H, Whp, g.eta, wv.l0, wv.f0, wv.nf, wv.nv, scale, g.twW,                    \
                        const_cast<signed char*>(code), tpart);                                                      \
    return launch_pdl(k_wrow_vstep<N, 1>, dim3(ctas), dim3(RowGeo<N>::NTH), vstep_smem<N, 1>(), st, Y, bvbar, thr, \
                      g.ranges, g.H, Whp, g.eta, wv.l0, wv.f0, wv.nf, wv.nv, scale, g.twW,                        \
                      const_cast<signed char*>(code), tpart);
    SHF_FAST_SIZES(SHF_CASE)
#undef SHF_CASE
    default: return cudaErrorInvalidValue;
  }
}

size_t ustep_smem_bytes(int L, int K) {
  switch (L) {
#define SHF_CASE(N) \
  case N:           \
    return ustep_smem<N>(K);
    SHF_FAST_SIZES(SHF_CASE)
#undef SHF_CASE
    default: return 0;
  }
}

cudaError_t row_ustep(const Geo& g, const float2* T, const float* s, float* w, float* bw, float* u, float2* Ur, int K,
                      float gamma, float scale, cudaStream_t st) {
  switch (g.L) {
#define SHF_CASE(N) \
  case N:           \
    return ustep_t<N>(g, T, s, w, bw, u, Ur, K, gamma, scale, st);
    SHF_FAST_SIZES(SHF_CASE)
#undef SHF_CASE
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fast
}  // namespace shf

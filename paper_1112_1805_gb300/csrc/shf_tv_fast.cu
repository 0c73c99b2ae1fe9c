// The u-step of the TV model (Sec. 4, eq. TVreg) on register FFTs for
// power-of-two sizes (half width L = W/2 in 64..1024, H in 512, 1024, 2048):
// (I + grad^T grad) u = rhs solved as u = ifft2(fft2(rhs) / symbol) with
// three kernels that keep each transform in registers,
//   rows_fwd: rhs = q + grad^T d formed per row (periodic backward
//             differences of d), the real row transformed as a packed complex
//             row of length L (radix-16 passes, 16 values per thread), the
//             half spectrum [0, L] unpacked and stored;
//   cols:     per column tile of the half spectrum: forward column transform,
//             division by the symbol 1 + 4 sin^2(pi n1/H) + 4 sin^2(pi n2/W)
//             (multiplication by its stored inverse), inverse transform;
//   rows_inv: inverse packing, inverse row transform, scaled by 1/(H W) into u.
// The packing pairs X_n with X_{L-n} and the unpacking Z_i with Z_{L-i} as in
// the shearlet v-step (partner-lane shuffles for groups of up to 32 threads;
// for L = 1024 the partner values come from L2 and the exchange buffer).
#include <algorithm>

#include "shf_fast.h"
#include "shf_fft16.cuh"

namespace shf {
namespace tvfast {
namespace {

using fast::launch_pdl;
using fast::load_table;
using fast::pdl_trigger;
using fast::pdl_wait;

__host__ __device__ constexpr int even2(int n) { return (n + 1) & ~1; }
__host__ __device__ constexpr bool row_len_ok(int L) { return L == 64 || L == 128 || L == 256 || L == 512 || L == 1024; }
__host__ __device__ constexpr bool col_len_ok(int H) { return H == 512 || H == 1024 || H == 2048; }

// Row groups of T = L/16 threads: 32/T groups per warp (T <= 32) or T/32
// warps per group, eight warps per CTA; per group the FFT exchange buffer,
// groups of a half-warp T float2 apart modulo 16 in the banks.
template <int L>
struct RowGeo {
  static constexpr int T = L / 16;
  static constexpr int RPC = T <= 32 ? 8 * (32 / T) : 256 / T;
  static constexpr int BUF = even2(reg::row_buf(L));
  static constexpr int STRIDE = T >= 16 ? BUF : BUF + ((T - BUF % 16) % 16 + 16) % 16;
  static constexpr int TW = even2(L + 1);
  static constexpr int PT = even2(r16::Passes<L>::TWSIZE);
  static constexpr int TOTAL = TW + PT + RPC * STRIDE;  // float2 per CTA
};

template <int H>
struct ColGeo {
  static constexpr int KB = reg::col_batch(H);
  static constexpr int T = H / 16;
  static constexpr int NT = KB * T;
  static constexpr int PT = even2(r16::Passes<H>::TWSIZE);
  static constexpr int BR = r16::brows16(H) * KB;
  static constexpr int TOTAL = PT + 2 * BR;
};

template <int L>
__global__ void __launch_bounds__(256, 2)
    k_tv_rows_fwd(const float* __restrict__ q, const float* __restrict__ d, float2* __restrict__ Ur, int K, int H,
                  int Whp, const float2* __restrict__ twW) {
  using G = RowGeo<L>;
  constexpr int T = G::T, RPC = G::RPC, W = 2 * L;
  extern __shared__ __align__(16) float2 sm[];
  float2* tw = sm;
  float2* pt = tw + G::TW;
  const int lane = threadIdx.x & 31;
  const int tt = threadIdx.x & (T - 1);
  const int grp = threadIdx.x / T;
  const int partner = T <= 32 ? (lane - tt) + ((T - tt) & (T - 1)) : 0;
  const int bar = 1 + grp;
  float2* fb = pt + G::PT + grp * G::STRIDE;
  load_table(tw, twW, L + 1);
  r16::build_pass_twiddles<L, 2>(pt, twW, threadIdx.x, blockDim.x);
  pdl_wait();
  pdl_trigger();
  __syncthreads();
  const size_t P = static_cast<size_t>(H) * W;
  const int rows = K * H, Gn = gridDim.x * RPC, gid = blockIdx.x * RPC + grp;
  const int niter = (rows + Gn - 1) / Gn;  // the same for every group: every lane takes part in the shuffles
  for (int it = 0; it < niter; ++it) {
    const int rr = gid + it * Gn;
    const bool live = rr < rows;
    const int r = live ? rr : 0;
    const int k = r / H, row = r - k * H, rowm = row == 0 ? H - 1 : row - 1;
    const float* qr = q + k * P + static_cast<size_t>(row) * W;
    const float* d0 = d + 2 * k * P;
    const float* d0r = d0 + static_cast<size_t>(row) * W;
    const float* d0m = d0 + static_cast<size_t>(rowm) * W;
    const float* d1r = d0 + P + static_cast<size_t>(row) * W;
    float2 v[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int c = 2 * (tt + j * T);
      const float2 qq = *reinterpret_cast<const float2*>(qr + c);
      const float2 a = *reinterpret_cast<const float2*>(d0r + c);
      const float2 am = *reinterpret_cast<const float2*>(d0m + c);
      const float2 b = *reinterpret_cast<const float2*>(d1r + c);
      const float bm = d1r[c == 0 ? W - 1 : c - 1];
      v[j] = live ? make_float2(qq.x + ((am.x - a.x) + (bm - b.x)), qq.y + ((am.y - a.y) + (b.x - b.y)))
                  : make_float2(0.f, 0.f);
    }
    r16::row_fft<L, -1>(v, tt, fb, pt, bar);
    float2* X = Ur + static_cast<size_t>(r) * Whp;
    if constexpr (T <= 32) {
#pragma unroll
      for (int qi = 0; qi < 16; ++qi) {
        float2 pr;
        pr.x = __shfl_sync(0xffffffffu, v[15 - qi].x, partner);
        pr.y = __shfl_sync(0xffffffffu, v[15 - qi].y, partner);
        const float2 x = r16::unpack_value<L>(v, qi, tt, pr, tw);
        if (live) X[tt + qi * T] = x;
      }
    } else {
      r16::group_sync<L>(bar);  // the last pass may still read the buffer
#pragma unroll
      for (int qi = 0; qi < 16; ++qi) fb[reg::ridx(tt + qi * T)] = v[qi];
      r16::group_sync<L>(bar);
#pragma unroll
      for (int qi = 0; qi < 16; ++qi) {
        const int i = tt + qi * T;
        const float2 x = r16::unpack_value<L>(v, qi, tt, fb[reg::ridx((L - i) & (L - 1))], tw);
        if (live) X[i] = x;
      }
    }
    if (live && tt == 0) X[L] = make_float2(v[0].x - v[0].y, 0.f);  // i = L: e^{-i pi} = -1
  }
}

template <int L>
__global__ void __launch_bounds__(256, 2)
    k_tv_rows_inv(const float2* __restrict__ Y, float* __restrict__ u, int K, int H, int Whp, float scale,
                  const float2* __restrict__ twW) {
  using G = RowGeo<L>;
  constexpr int T = G::T, RPC = G::RPC, W = 2 * L;
  extern __shared__ __align__(16) float2 sm[];
  float2* tw = sm;
  float2* pt = tw + G::TW;
  const int lane = threadIdx.x & 31;
  const int tt = threadIdx.x & (T - 1);
  const int grp = threadIdx.x / T;
  const int partner = T <= 32 ? (lane - tt) + ((T - tt) & (T - 1)) : 0;
  const int bar = 1 + grp;
  float2* fb = pt + G::PT + grp * G::STRIDE;
  load_table(tw, twW, L + 1);
  r16::build_pass_twiddles<L, 2>(pt, twW, threadIdx.x, blockDim.x);
  pdl_wait();
  pdl_trigger();
  __syncthreads();
  const int rows = K * H, Gn = gridDim.x * RPC, gid = blockIdx.x * RPC + grp;
  const int niter = (rows + Gn - 1) / Gn;
  for (int it = 0; it < niter; ++it) {
    const int rr = gid + it * Gn;
    const bool live = rr < rows;
    const int r = live ? rr : 0;
    const float2* X = Y + static_cast<size_t>(r) * Whp;
    float2 v[16];
    if constexpr (T <= 32) {
      // inverse packing (r16::pack_step), X_{L-n} from the partner lane
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = __ldcg(X + tt + j * T);
      float2 prev = __ldcg(X + L);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        float2 ra, rb;
        ra.x = __shfl_sync(0xffffffffu, v[15 - j].x, partner);
        ra.y = __shfl_sync(0xffffffffu, v[15 - j].y, partner);
        rb.x = __shfl_sync(0xffffffffu, v[j].x, partner);
        rb.y = __shfl_sync(0xffffffffu, v[j].y, partner);
        r16::pack_step<L>(v, j, tt, ra, rb, prev, tw);
      }
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int n = tt + j * T, m = L - n;
        const float2 a = __ldcg(X + n);
        const float2 c = c_conj(__ldcg(X + m));
        const float2 s2 = c_add(a, c), dd = c_sub(a, c);
        v[j] = pack_combine(s2, dd, tw[n]);
      }
    }
    r16::row_fft<L, +1>(v, tt, fb, pt, bar);
    if (live) {
      float* ur = u + static_cast<size_t>(r) * W;
#pragma unroll
      for (int j = 0; j < 16; ++j)
        *reinterpret_cast<float2*>(ur + 2 * (tt + j * T)) = make_float2(scale * v[j].x, scale * v[j].y);
    }
  }
}

template <int H>
__global__ void __launch_bounds__(ColGeo<H>::NT, H == 512 ? 2 : 1)
    k_tv_cols(const float2* __restrict__ Ur, const float* __restrict__ sym, float2* __restrict__ Y, int K, int Wh,
              int Whp, const float2* __restrict__ twH) {
  using G = ColGeo<H>;
  constexpr int KB = G::KB, T = G::T;
  extern __shared__ __align__(16) float2 sm[];
  float2* pt = sm;
  float2* b0 = sm + G::PT;
  float2* b1 = b0 + G::BR;
  const int b = threadIdx.x % KB, tt = threadIdx.x / KB;
  r16::build_pass_twiddles<H, 1>(pt, twH, threadIdx.x, blockDim.x);
  pdl_wait();
  pdl_trigger();
  const int ntiles = (Wh + KB - 1) / KB, items = K * ntiles;
  for (int item = blockIdx.x; item < items; item += gridDim.x) {
    const int k = item / ntiles, col = (item - k * ntiles) * KB + b;
    const bool ok = col < Wh;
    const float2* src = Ur + static_cast<size_t>(k) * H * Whp + col;
    float2 v[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = ok ? src[static_cast<size_t>(tt + j * T) * Whp] : make_float2(0.f, 0.f);
    r16::batch_fft<H, -1, KB>(v, tt, b, b0, b1, pt);  // starts with a CTA barrier
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = c_scale(v[j], ok ? sym[static_cast<size_t>(tt + j * T) * Wh + col] : 0.f);
    r16::batch_fft<H, +1, KB>(v, tt, b, b0, b1, pt);
    if (ok) {
      float2* dst = Y + static_cast<size_t>(k) * H * Whp + col;
#pragma unroll
      for (int j = 0; j < 16; ++j) dst[static_cast<size_t>(tt + j * T) * Whp] = v[j];
    }
  }
}

template <int L>
size_t row_smem() {
  return sizeof(float2) * RowGeo<(row_len_ok(L) ? L : 64)>::TOTAL;
}
template <int H>
size_t col_smem() {
  return sizeof(float2) * ColGeo<(col_len_ok(H) ? H : 512)>::TOTAL;
}

int resident(const void* kernel, int threads, size_t smem) {
  int dev = 0, sms = 0, fit = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, kernel, threads, smem) != cudaSuccess) return 0;
  return fit * sms;
}

}  // namespace

bool tv_fast_ok(int H, int W) { return col_len_ok(H) && row_len_ok(W / 2) && W % 2 == 0; }

int tv_fast_pitch(int W) { return (W / 2 + 1 + 7) & ~7; }

cudaError_t tv_fast_prepare() {
  cudaError_t e = cudaSuccess;
#define SHF_TV_ROW(N)                                                             \
  if (e == cudaSuccess) e = fast::allow_smem(k_tv_rows_fwd<N>, row_smem<N>());   \
  if (e == cudaSuccess) e = fast::allow_smem(k_tv_rows_inv<N>, row_smem<N>());
  SHF_TV_ROW(64) SHF_TV_ROW(128) SHF_TV_ROW(256) SHF_TV_ROW(512) SHF_TV_ROW(1024)
#undef SHF_TV_ROW
#define SHF_TV_COL(N) \
  if (e == cudaSuccess) e = fast::allow_smem(k_tv_cols<N>, col_smem<N>());
  SHF_TV_COL(512) SHF_TV_COL(1024) SHF_TV_COL(2048)
#undef SHF_TV_COL
  return e;
}

cudaError_t tv_fast_rows_fwd(const float* q, const float* d, float2* Ur, int K, int H, int W, const float2* twW,
                             cudaStream_t st) {
  const int Whp = tv_fast_pitch(W);
  switch (W / 2) {
#define SHF_CASE(N)                                                                                              \
  case N: {                                                                                                      \
    const int ctas = std::min(resident(reinterpret_cast<const void*>(k_tv_rows_fwd<N>), 256, row_smem<N>()),   \
                              (K * H + RowGeo<N>::RPC - 1) / RowGeo<N>::RPC);                                  \
    return launch_pdl(k_tv_rows_fwd<N>, dim3(std::max(ctas, 1)), dim3(256), row_smem<N>(), st, q, d, Ur, K, H,  \
                      Whp, twW);                                                                                 \
  }
    SHF_CASE(64) SHF_CASE(128) SHF_CASE(256) SHF_CASE(512) SHF_CASE(1024)
#undef SHF_CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t tv_fast_rows_inv(const float2* Y, float* u, int K, int H, int W, float scale, const float2* twW,
                             cudaStream_t st) {
  const int Whp = tv_fast_pitch(W);
  switch (W / 2) {
#define SHF_CASE(N)                                                                                              \
  case N: {                                                                                                      \
    const int ctas = std::min(resident(reinterpret_cast<const void*>(k_tv_rows_inv<N>), 256, row_smem<N>()),   \
                              (K * H + RowGeo<N>::RPC - 1) / RowGeo<N>::RPC);                                  \
    return launch_pdl(k_tv_rows_inv<N>, dim3(std::max(ctas, 1)), dim3(256), row_smem<N>(), st, Y, u, K, H, Whp, \
                      scale, twW);                                                                               \
  }
    SHF_CASE(64) SHF_CASE(128) SHF_CASE(256) SHF_CASE(512) SHF_CASE(1024)
#undef SHF_CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t tv_fast_cols(const float2* Ur, const float* sym, float2* Y, int K, int H, int W, const float2* twH,
                         cudaStream_t st) {
  const int Wh = W / 2 + 1, Whp = tv_fast_pitch(W);
  switch (H) {
#define SHF_CASE(N)                                                                                             \
  case N: {                                                                                                     \
    const int items = K * ((Wh + ColGeo<N>::KB - 1) / ColGeo<N>::KB);                                          \
    const int ctas = std::min(resident(reinterpret_cast<const void*>(k_tv_cols<N>), ColGeo<N>::NT, col_smem<N>()), \
                              items);                                                                           \
    return launch_pdl(k_tv_cols<N>, dim3(std::max(ctas, 1)), dim3(ColGeo<N>::NT), col_smem<N>(), st, Ur, sym, Y, \
                      K, Wh, Whp, twH);                                                                         \
  }
    SHF_CASE(512) SHF_CASE(1024) SHF_CASE(2048)
#undef SHF_CASE
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace tvfast
}  // namespace shf

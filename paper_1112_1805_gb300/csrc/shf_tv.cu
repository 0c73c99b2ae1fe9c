// TV-regularised segmentation, the comparison model of Sec. 4 (eq. TVreg):
//   min_u <u, s> + lambda || |(I_q (x) grad) u| ||_1 + iota_C(u),
// solved by the ADMM of Sec. 3 with the shearlet transform S replaced by the
// gradient: splitting v = (I_q (x) grad) u, w = u, and per iteration
//   u   = (I + grad^T grad)^(-1) [ grad^T (v - b_v) + (w - b_w) - gamma s ]
//   v   = group shrinkage of g = b_v + grad u by gamma lambda, b_v = g - v
//   w   = pixelwise projection of g_w = b_w + u onto the simplex, b_w = g_w - w.
// grad is the forward difference with periodic boundary (the periodic setting
// of the FFT-based shearlets), so I + grad^T grad is diagonal in the DFT basis
// with symbol 1 + 4 sin^2(pi n1/H) + 4 sin^2(pi n2/W): the u-step is one
// filtered 2-D FFT per label, run by the general transform kernels with that
// symbol as a one-filter bank.  The group of the shrinkage is all 2K values
// of a pixel (the labels coupled, as eq. TVreg writes it) or the two values of
// each label (the alternative the paper mentions).
//
// State per iteration, as in the shearlet path: only b_v is kept of the pair
// (v, b_v), with d = v - b_v = g - 2 b_v feeding the next right-hand side.
#include <cmath>
#include <string>
#include <vector>

#include "shearseg.h"
#include "shf_internal.h"
#include "shf_simplex.cuh"

using shf::Geo;

struct tv_state {
  Geo g;  // eta = 1: the filter is the inverse symbol of I + grad^T grad
  int K = 0, C = 0, per_label = 0, device = 0;
  bool fast = false;  // register-FFT u-step (power-of-two sizes), spectra at row pitch `pitch`
  int pitch = 0;
  float gamma = 1.f, lambda = 0.f;
  std::vector<float> codebook;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  float *f = nullptr, *s = nullptr, *u = nullptr, *bv = nullptr, *d = nullptr, *w = nullptr, *bw = nullptr;
  float *q = nullptr, *rhs = nullptr, *sym = nullptr, *gap = nullptr;
  float2 *twH = nullptr, *twW = nullptr, *Ur = nullptr, *Y = nullptr;
  int* labels = nullptr;
  int* flag = nullptr;
  double* red = nullptr;
  int iter = 0;
  cudaGraphExec_t exec = nullptr;
  bool graph_tried = false;
  size_t P() const { return static_cast<size_t>(g.H) * g.W; }
};

namespace {

constexpr int kThreads = 256;
constexpr int kRedBlocks = 512;
constexpr double kPi = 3.14159265358979323846;

// 1 / (1 + 4 sin^2(pi n1 / H) + 4 sin^2(pi n2 / W)) on the half plane [H][W/2+1].
__global__ void k_poisson_symbol(float* __restrict__ sym, int H, int W, int Wh) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= H * Wh) return;
  const int n1 = i / Wh, n2 = i - n1 * Wh;
  const double s1 = sin(kPi * n1 / H), s2 = sin(kPi * n2 / W);
  sym[i] = static_cast<float>(1.0 / (1.0 + 4.0 * s1 * s1 + 4.0 * s2 * s2));
}

// The v-, w- and b-updates after the u-step, per pixel over the K labels:
// g = b_v + grad u (forward differences, periodic), b_v <- g min(1, t/|g|)
// (the group clip; v = g - b_v is the shrinkage), d = g - 2 b_v;
// g_w = b_w + u, w = P_C(g_w), b_w = g_w - w; q = (w - b_w) - gamma s.
template <int KM>
__global__ void __launch_bounds__(kThreads) k_tv_prox(const float* __restrict__ u, float* __restrict__ bv,
                                                      float* __restrict__ d, float* __restrict__ w,
                                                      float* __restrict__ bw, const float* __restrict__ s,
                                                      float* __restrict__ q, int K, int H, int W, float t,
                                                      float gamma, int per_label) {
  const size_t P = static_cast<size_t>(H) * W;
  for (size_t x = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; x < P;
       x += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const int r = static_cast<int>(x / W), c = static_cast<int>(x - static_cast<size_t>(r) * W);
    const size_t xr = static_cast<size_t>(r + 1 == H ? 0 : r + 1) * W + c;  // next row
    const size_t xc = static_cast<size_t>(r) * W + (c + 1 == W ? 0 : c + 1);  // next column
    float uk[KM], g0[KM], g1[KM];
    float n2 = 0.f;
#pragma unroll
    for (int k = 0; k < KM; ++k) {
      if (k < K) {
        const float* up = u + k * P;
        uk[k] = up[x];
        g0[k] = bv[(2 * k) * P + x] + (up[xr] - uk[k]);
        g1[k] = bv[(2 * k + 1) * P + x] + (up[xc] - uk[k]);
        n2 = fmaf(g0[k], g0[k], n2);
        n2 = fmaf(g1[k], g1[k], n2);
      }
    }
    const float nall = sqrtf(n2);
    const float fall = nall > t ? t / nall : 1.f;
#pragma unroll
    for (int k = 0; k < KM; ++k) {
      if (k < K) {
        float fk = fall;
        if (per_label) {
          const float nk = sqrtf(fmaf(g0[k], g0[k], g1[k] * g1[k]));
          fk = nk > t ? t / nk : 1.f;
        }
        const float b0 = fk * g0[k], b1 = fk * g1[k];
        bv[(2 * k) * P + x] = b0;
        bv[(2 * k + 1) * P + x] = b1;
        d[(2 * k) * P + x] = g0[k] - 2.f * b0;
        d[(2 * k + 1) * P + x] = g1[k] - 2.f * b1;
      }
    }
    float gw[KM];
#pragma unroll
    for (int k = 0; k < KM; ++k) gw[k] = k < K ? bw[k * P + x] + uk[k] : 0.f;
    float wk[KM];
#pragma unroll
    for (int k = 0; k < KM; ++k) wk[k] = gw[k];
    shf::simplex_project<KM>(wk, K);
#pragma unroll
    for (int k = 0; k < KM; ++k) {
      if (k < K) {
        const float bn = gw[k] - wk[k];
        w[k * P + x] = wk[k];
        bw[k * P + x] = bn;
        q[k * P + x] = (wk[k] - bn) - gamma * s[k * P + x];
      }
    }
  }
}

// rhs = q + grad^T d: (grad^T d)(r, c) = d0(r-1, c) - d0(r, c) + d1(r, c-1) - d1(r, c).
__global__ void __launch_bounds__(kThreads) k_tv_rhs(const float* __restrict__ q, const float* __restrict__ d,
                                                     float* __restrict__ rhs, int K, int H, int W) {
  const size_t P = static_cast<size_t>(H) * W;
  const size_t n = P * K;
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const size_t k = i / P, x = i - k * P;
    const int r = static_cast<int>(x / W), c = static_cast<int>(x - static_cast<size_t>(r) * W);
    const float* d0 = d + 2 * k * P;
    const float* d1 = d0 + P;
    const size_t xr = static_cast<size_t>(r == 0 ? H - 1 : r - 1) * W + c;
    const size_t xc = static_cast<size_t>(r) * W + (c == 0 ? W - 1 : c - 1);
    rhs[i] = q[i] + ((d0[xr] - d0[x]) + (d1[xc] - d1[x]));
  }
}

// q = (w - b_w) - gamma s (after w or b_w were set from outside; -gamma s at
// the zero state).
__global__ void k_tv_q(const float* __restrict__ w, const float* __restrict__ bw, const float* __restrict__ s,
                       float* __restrict__ q, float gamma, size_t n) {
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * blockDim.x)
    q[i] = (w[i] - bw[i]) - gamma * s[i];
}

// out = a + sb b (v = d + b_v for the readout; d = v - b_v in place, so out
// may alias a).
__global__ void k_axpb(const float* a, const float* __restrict__ b, float* out, float sb, size_t n) {
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * blockDim.x)
    out[i] = a[i] + sb * b[i];
}

// Energy partials in FP64: per block, sum over its pixels (fixed order) of
// <w, s> at the pixel and lambda |(I_q (x) grad) w|(pixel); partial[2 block]
// and partial[2 block + 1].
__global__ void __launch_bounds__(kThreads) k_tv_energy(const float* __restrict__ w, const float* __restrict__ s,
                                                        int K, int H, int W, int per_label,
                                                        double* __restrict__ partial) {
  const size_t P = static_cast<size_t>(H) * W;
  double ds = 0.0, dt = 0.0;
  for (size_t x = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; x < P;
       x += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const int r = static_cast<int>(x / W), c = static_cast<int>(x - static_cast<size_t>(r) * W);
    const size_t xr = static_cast<size_t>(r + 1 == H ? 0 : r + 1) * W + c;
    const size_t xc = static_cast<size_t>(r) * W + (c + 1 == W ? 0 : c + 1);
    double n2 = 0.0;
    for (int k = 0; k < K; ++k) {
      const float* wp = w + k * P;
      const double a = static_cast<double>(wp[xr]) - wp[x], b = static_cast<double>(wp[xc]) - wp[x];
      ds += static_cast<double>(wp[x]) * s[k * P + x];
      if (per_label)
        dt += sqrt(a * a + b * b);
      else
        n2 += a * a + b * b;
    }
    if (!per_label) dt += sqrt(n2);
  }
  __shared__ double sh[2][kThreads];
  sh[0][threadIdx.x] = ds;
  sh[1][threadIdx.x] = dt;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + o];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = sh[0][0];
    partial[2 * blockIdx.x + 1] = sh[1][0];
  }
}

// out[0] = sum of the even partials, out[1] = sum of the odd ones, in order.
__global__ void k_tv_energy_final(const double* __restrict__ partial, int nblocks, double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double a = 0.0, b = 0.0;
  for (int i = 0; i < nblocks; ++i) {
    a += partial[2 * i];
    b += partial[2 * i + 1];
  }
  out[0] = a;
  out[1] = b;
}

int tv_fail(int code, const std::string& msg) { return shf::set_error(code, msg); }

#define TV_CK(call)                                                                                        \
  do {                                                                                                     \
    cudaError_t e_ = (call);                                                                               \
    if (e_ != cudaSuccess) return tv_fail(SHF_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <typename T>
int tv_alloc(T** p, size_t count, const char* what) {
  *p = nullptr;
  if (count == 0) return SHF_OK;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return tv_fail(e == cudaErrorMemoryAllocation ? SHF_ERR_OOM : SHF_ERR_CUDA,
                   std::string("cudaMalloc(") + what + "): " + cudaGetErrorString(e));
  }
  return SHF_OK;
}

int grid_for(size_t n) {
  const size_t b = (n + kThreads - 1) / kThreads;
  return static_cast<int>(b < 8192 ? (b ? b : 1) : 8192);
}

void free_tv(tv_state* st) {
  if (!st) return;
  if (st->stream) cudaStreamSynchronize(st->stream);
  if (st->exec) cudaGraphExecDestroy(st->exec);
  void* bufs[] = {st->f, st->s, st->u, st->bv, st->d, st->w, st->bw, st->q, st->rhs, st->sym, st->gap,
                  st->twH, st->twW, st->Ur, st->Y, st->labels, st->flag, st->red};
  for (void* b : bufs) cudaFree(b);
  if (st->own_stream && st->stream) cudaStreamDestroy(st->stream);
  delete st;
}

// Kernels of one iteration, in order (for tv_admm_kernel_times).
enum TvKind { kTvRowFwd = 0, kTvCol = 1, kTvRowInv = 2, kTvProx = 3, kTvRhs = 4, kTvKinds = 5 };
const char* const kTvNames[kTvKinds] = {"tv_row_fwd", "tv_col_solve", "tv_row_inv", "tv_prox", "tv_rhs"};

cudaError_t launch_prox(tv_state* st) {
  const Geo& g = st->g;
  const size_t P = st->P();
  const float t = st->gamma * st->lambda;
  const int grid = grid_for(P);
  if (st->K <= 4)
    k_tv_prox<4><<<grid, kThreads, 0, st->stream>>>(st->u, st->bv, st->d, st->w, st->bw, st->s, st->q, st->K, g.H,
                                                     g.W, t, st->gamma, st->per_label);
  else if (st->K <= 8)
    k_tv_prox<8><<<grid, kThreads, 0, st->stream>>>(st->u, st->bv, st->d, st->w, st->bw, st->s, st->q, st->K, g.H,
                                                     g.W, t, st->gamma, st->per_label);
  else
    k_tv_prox<16><<<grid, kThreads, 0, st->stream>>>(st->u, st->bv, st->d, st->w, st->bw, st->s, st->q, st->K,
                                                      g.H, g.W, t, st->gamma, st->per_label);
  return cudaGetLastError();
}

cudaError_t launch_rhs(tv_state* st) {
  k_tv_rhs<<<grid_for(st->P() * st->K), kThreads, 0, st->stream>>>(st->q, st->d, st->rhs, st->K, st->g.H, st->g.W);
  return cudaGetLastError();
}

// One iteration; `ev` (nullable, kTvKinds + 1 events) is recorded before each
// launch and after the last.
cudaError_t enqueue_tv_iteration(tv_state* st, cudaEvent_t* ev) {
  const Geo& g = st->g;
  cudaStream_t ss = st->stream;
  auto mark = [&](int i) { return ev ? cudaEventRecord(ev[i], ss) : cudaSuccess; };
  // plain stream order: with programmatic dependent launch the 512 x 512
  // iteration measured 3.8% slower
  const shf::PdlScope pdl(false);
  if (st->fast) {  // the right-hand side is formed inside the row transforms
    const float scale = 1.f / (static_cast<float>(g.H) * g.W);
    cudaError_t e = mark(kTvRowFwd);
    if (e == cudaSuccess) e = shf::tvfast::tv_fast_rows_fwd(st->q, st->d, st->Ur, st->K, g.H, g.W, g.twW, ss);
    if (e == cudaSuccess) e = mark(kTvCol);
    if (e == cudaSuccess) e = shf::tvfast::tv_fast_cols(st->Ur, st->sym, st->Y, st->K, g.H, g.W, g.twH, ss);
    if (e == cudaSuccess) e = mark(kTvRowInv);
    if (e == cudaSuccess) e = shf::tvfast::tv_fast_rows_inv(st->Y, st->u, st->K, g.H, g.W, scale, g.twW, ss);
    if (e == cudaSuccess) e = mark(kTvProx);
    if (e == cudaSuccess) e = launch_prox(st);
    if (e == cudaSuccess) e = mark(kTvRhs);
    if (e == cudaSuccess) e = mark(kTvKinds);
    return e;
  }
  cudaError_t e = mark(kTvRowFwd);
  if (e == cudaSuccess) e = shf::run_row_r2c(g, st->rhs, st->Ur, st->K, 1.f, ss);
  if (e == cudaSuccess) e = mark(kTvCol);
  if (e == cudaSuccess) e = shf::run_col_fan(g, st->Ur, st->Y, st->K, 1, ss);
  if (e == cudaSuccess) e = mark(kTvRowInv);
  if (e == cudaSuccess) e = shf::run_row_c2r(g, st->Y, st->u, st->K, 1.f / (static_cast<float>(g.H) * g.W), ss);
  if (e == cudaSuccess) e = mark(kTvProx);
  if (e == cudaSuccess) e = launch_prox(st);
  if (e == cudaSuccess) e = mark(kTvRhs);
  if (e == cudaSuccess) e = launch_rhs(st);
  if (e == cudaSuccess) e = mark(kTvKinds);
  return e;
}

// rhs from the current (w, b_w, d): q = (w - b_w) - gamma s, rhs = q + grad^T d.
cudaError_t rebuild_rhs(tv_state* st) {
  const size_t n = st->P() * st->K;
  k_tv_q<<<grid_for(n), kThreads, 0, st->stream>>>(st->w, st->bw, st->s, st->q, st->gamma, n);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? launch_rhs(st) : e;
}

// Data term and the zero state v = b_v = w = b_w = 0.
int tv_restart(tv_state* st) {
  const size_t P = st->P(), K = st->K;
  TV_CK(shf::launch_count_nonfinite(st->f, static_cast<long>(P * st->C), st->flag, st->stream));
  int bad = 0;
  TV_CK(cudaMemcpyAsync(&bad, st->flag, sizeof(int), cudaMemcpyDeviceToHost, st->stream));
  TV_CK(cudaStreamSynchronize(st->stream));
  if (bad) return tv_fail(SHF_ERR_NONFINITE, "tv: the image contains NaN or Inf");
  TV_CK(shf::launch_data_term(st->f, st->C, st->codebook.data(), st->K, st->s, static_cast<int>(P), st->stream));
  TV_CK(cudaMemsetAsync(st->u, 0, sizeof(float) * P * K, st->stream));
  TV_CK(cudaMemsetAsync(st->w, 0, sizeof(float) * P * K, st->stream));
  TV_CK(cudaMemsetAsync(st->bw, 0, sizeof(float) * P * K, st->stream));
  TV_CK(cudaMemsetAsync(st->bv, 0, sizeof(float) * 2 * P * K, st->stream));
  TV_CK(cudaMemsetAsync(st->d, 0, sizeof(float) * 2 * P * K, st->stream));
  TV_CK(rebuild_rhs(st));
  TV_CK(cudaStreamSynchronize(st->stream));  // the codebook is read from host memory by the data term
  st->iter = 0;
  return SHF_OK;
}

int tv_copy(tv_state* st, void* dst, const void* src, size_t bytes, cudaMemcpyKind kind, bool sync) {
  TV_CK(cudaMemcpyAsync(dst, src, bytes, kind, st->stream));
  if (sync) TV_CK(cudaStreamSynchronize(st->stream));
  return SHF_OK;
}

}  // namespace

extern "C" {

int tv_admm_init(int H, int W, const float* f, int C, const float* codebook, int K, const tv_params* p,
                 void* stream, tv_state** out) {
  if (!out) return tv_fail(SHF_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!f || !codebook || !p) return tv_fail(SHF_ERR_ARG, "tv_admm_init: NULL argument");
  if (K < 2 || K > shf::kMaxK) return tv_fail(SHF_ERR_ARG, "K must be in [2, 16]");
  if (C != 1 && C != 3) return tv_fail(SHF_ERR_ARG, "C must be 1 or 3");
  if (!(p->gamma > 0.f) || !std::isfinite(p->gamma)) return tv_fail(SHF_ERR_ARG, "gamma must be positive and finite");
  if (!(p->lambda >= 0.f) || !std::isfinite(p->lambda))
    return tv_fail(SHF_ERR_ARG, "lambda must be finite and non-negative");
  if (reinterpret_cast<uintptr_t>(f) & 7u) return tv_fail(SHF_ERR_ARG, "f must be 8-byte aligned");
  if (H < 8 || W < 8 || H > shf::kMaxSide || W > shf::kMaxSide) return tv_fail(SHF_ERR_SIZE, "H and W must be in [8, 2048]");
  if (W & 1) return tv_fail(SHF_ERR_SIZE, "W must be even");
  for (int i = 0; i < K * C; ++i)
    if (!std::isfinite(codebook[i])) return tv_fail(SHF_ERR_NONFINITE, "codebook contains NaN or Inf");
  Geo g;
  if (!shf::make_geo(H, W, 1, &g)) return tv_fail(SHF_ERR_SIZE, "H and W/2 must be products of powers of 2, 3 and 5");
  g.eta = 1;
  int device = 0, optin = 0;
  TV_CK(cudaGetDevice(&device));
  TV_CK(shf::prepare_kernels());
  TV_CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
  if (shf::max_dynamic_smem_needed(g, K) > optin) return tv_fail(SHF_ERR_SIZE, "tile does not fit in shared memory");
  auto* st = new tv_state();
  st->K = K;
  st->C = C;
  st->device = device;
  st->gamma = p->gamma;
  st->lambda = p->lambda;
  st->per_label = p->per_label ? 1 : 0;
  st->codebook.assign(codebook, codebook + K * C);
  if (stream) {
    st->stream = static_cast<cudaStream_t>(stream);
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&st->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete st;
      return tv_fail(SHF_ERR_CUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
    }
    st->own_stream = true;
  }
  st->fast = shf::tvfast::tv_fast_ok(H, W);
  if (st->fast) {
    cudaError_t e = shf::tvfast::tv_fast_prepare();
    if (e != cudaSuccess) {
      free_tv(st);
      return tv_fail(SHF_ERR_CUDA, std::string("tv_admm_init: ") + cudaGetErrorString(e));
    }
  }
  st->pitch = st->fast ? shf::tvfast::tv_fast_pitch(W) : g.Wh;
  const size_t P = static_cast<size_t>(H) * W, Ph = static_cast<size_t>(H) * g.Wh;
  const size_t Phs = static_cast<size_t>(H) * st->pitch;  // spectra of the u-step at the path's pitch
  int rc;
  if ((rc = tv_alloc(&st->f, P * C, "f")) || (rc = tv_alloc(&st->s, P * K, "s")) ||
      (rc = tv_alloc(&st->u, P * K, "u")) || (rc = tv_alloc(&st->bv, 2 * P * K, "b_v")) ||
      (rc = tv_alloc(&st->d, 2 * P * K, "d")) || (rc = tv_alloc(&st->w, P * K, "w")) ||
      (rc = tv_alloc(&st->bw, P * K, "b_w")) || (rc = tv_alloc(&st->q, P * K, "q")) ||
      (rc = tv_alloc(&st->rhs, P * K, "rhs")) || (rc = tv_alloc(&st->sym, Ph, "symbol")) ||
      (rc = tv_alloc(&st->gap, P, "gap")) || (rc = tv_alloc(&st->twH, H, "twH")) ||
      (rc = tv_alloc(&st->twW, W, "twW")) || (rc = tv_alloc(&st->Ur, Phs * K, "Ur")) ||
      (rc = tv_alloc(&st->Y, Phs * K, "Y")) || (rc = tv_alloc(&st->labels, P, "labels")) ||
      (rc = tv_alloc(&st->flag, 1, "flag")) || (rc = tv_alloc(&st->red, 2 * kRedBlocks + 2, "red"))) {
    free_tv(st);
    return rc;
  }
  g.twH = st->twH;
  g.twW = st->twW;
  g.bank = st->sym;
  g.ranges = nullptr;
  st->g = g;
  cudaError_t e = shf::launch_twiddles(st->twH, H, st->stream);
  if (e == cudaSuccess) e = shf::launch_twiddles(st->twW, W, st->stream);
  if (e == cudaSuccess) {
    k_poisson_symbol<<<grid_for(Ph), kThreads, 0, st->stream>>>(st->sym, H, W, g.Wh);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(st->f, f, sizeof(float) * P * C, cudaMemcpyDeviceToDevice, st->stream);
  if (e != cudaSuccess) {
    free_tv(st);
    return tv_fail(SHF_ERR_CUDA, std::string("tv_admm_init: ") + cudaGetErrorString(e));
  }
  rc = tv_restart(st);
  if (rc) {
    free_tv(st);
    return rc;
  }
  *out = st;
  return SHF_OK;
}

int tv_admm_reset(tv_state* st, const float* f, int f_on_host) {
  if (!st || !f) return tv_fail(SHF_ERR_ARG, "tv_admm_reset: NULL argument");
  if (!f_on_host && (reinterpret_cast<uintptr_t>(f) & 7u)) return tv_fail(SHF_ERR_ARG, "f must be 8-byte aligned");
  TV_CK(cudaMemcpyAsync(st->f, f, sizeof(float) * st->P() * st->C,
                        f_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st->stream));
  return tv_restart(st);
}

int tv_admm_step(tv_state* st, int n) {
  if (!st || n < 0) return tv_fail(SHF_ERR_ARG, "tv_admm_step: bad argument");
  if (n == 0) return SHF_OK;
  if (!st->graph_tried) {
    // one iteration captured as a CUDA graph when the stream allows capture
    st->graph_tried = true;
    cudaGraph_t graph = nullptr;
    if (st->stream && cudaStreamBeginCapture(st->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      cudaError_t e = enqueue_tv_iteration(st, nullptr);
      cudaError_t e2 = cudaStreamEndCapture(st->stream, &graph);
      if (e == cudaSuccess && e2 == cudaSuccess && graph) {
        if (cudaGraphInstantiate(&st->exec, graph, 0) != cudaSuccess) st->exec = nullptr;
      }
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
    }
  }
  for (int i = 0; i < n; ++i) {
    if (st->exec)
      TV_CK(cudaGraphLaunch(st->exec, st->stream));
    else
      TV_CK(enqueue_tv_iteration(st, nullptr));
  }
  st->iter += n;
  return SHF_OK;
}

int tv_admm_kernel_times(tv_state* st, int n, float* ms, int* nk) {
  if (!st || !ms || n < 1) return tv_fail(SHF_ERR_ARG, "tv_admm_kernel_times: bad argument");
  cudaEvent_t ev[kTvKinds + 1];
  for (int i = 0; i <= kTvKinds; ++i) TV_CK(cudaEventCreate(&ev[i]));
  for (int i = 0; i < kTvKinds; ++i) ms[i] = 0.f;
  int rc = SHF_OK;
  for (int it = 0; it < n && rc == SHF_OK; ++it) {
    cudaError_t e = enqueue_tv_iteration(st, ev);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[kTvKinds]);
    for (int i = 0; i < kTvKinds && e == cudaSuccess; ++i) {
      float t = 0.f;
      e = cudaEventElapsedTime(&t, ev[i], ev[i + 1]);
      ms[i] += t / n;
    }
    if (e != cudaSuccess) rc = tv_fail(SHF_ERR_CUDA, std::string("tv_admm_kernel_times: ") + cudaGetErrorString(e));
  }
  for (int i = 0; i <= kTvKinds; ++i) cudaEventDestroy(ev[i]);
  if (rc == SHF_OK) st->iter += n;
  if (nk) *nk = kTvKinds;
  return rc;
}

const char* tv_admm_kernel_name(int i) { return (i >= 0 && i < kTvKinds) ? kTvNames[i] : ""; }

int tv_admm_get(tv_state* st, int what, void* dst, int on_host) {
  if (!st || !dst) return tv_fail(SHF_ERR_ARG, "tv_admm_get: NULL argument");
  const size_t P = st->P(), K = st->K;
  const cudaMemcpyKind kind = on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  switch (what) {
    case SEG_U: return tv_copy(st, dst, st->u, sizeof(float) * P * K, kind, on_host);
    case SEG_W: return tv_copy(st, dst, st->w, sizeof(float) * P * K, kind, on_host);
    case SEG_BW: return tv_copy(st, dst, st->bw, sizeof(float) * P * K, kind, on_host);
    case SEG_S: return tv_copy(st, dst, st->s, sizeof(float) * P * K, kind, on_host);
    case SEG_BV: return tv_copy(st, dst, st->bv, sizeof(float) * 2 * P * K, kind, on_host);
    case SEG_V: {  // v = d + b_v
      const size_t n = 2 * P * K;
      float* tgt = static_cast<float*>(dst);
      if (on_host) TV_CK(cudaMallocAsync(reinterpret_cast<void**>(&tgt), sizeof(float) * n, st->stream));
      k_axpb<<<grid_for(n), kThreads, 0, st->stream>>>(st->d, st->bv, tgt, 1.f, n);
      cudaError_t e = cudaGetLastError();
      if (on_host) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(dst, tgt, sizeof(float) * n, cudaMemcpyDeviceToHost, st->stream);
        cudaError_t e2 = cudaFreeAsync(tgt, st->stream);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaStreamSynchronize(st->stream);
      }
      TV_CK(e);
      return SHF_OK;
    }
    case SEG_LABELS:
    case SEG_GAP: {
      TV_CK(shf::launch_labels(st->w, st->K, static_cast<int>(P), st->labels, st->gap, st->stream));
      return tv_copy(st, dst, what == SEG_LABELS ? static_cast<void*>(st->labels) : static_cast<void*>(st->gap),
                     sizeof(float) * P, kind, on_host);
    }
    case SEG_ENERGY: {
      k_tv_energy<<<kRedBlocks, kThreads, 0, st->stream>>>(st->w, st->s, st->K, st->g.H, st->g.W, st->per_label,
                                                           st->red + 2);
      TV_CK(cudaGetLastError());
      k_tv_energy_final<<<1, 32, 0, st->stream>>>(st->red + 2, kRedBlocks, st->red);
      TV_CK(cudaGetLastError());
      double h[2];
      TV_CK(cudaMemcpyAsync(h, st->red, sizeof(h), cudaMemcpyDeviceToHost, st->stream));
      TV_CK(cudaStreamSynchronize(st->stream));
      const double energy = h[0] + static_cast<double>(st->lambda) * h[1];
      if (on_host) {
        *static_cast<double*>(dst) = energy;
        return SHF_OK;
      }
      return tv_copy(st, dst, &energy, sizeof(double), cudaMemcpyHostToDevice, true);
    }
    case SEG_ITER: {
      if (!on_host) return tv_fail(SHF_ERR_ARG, "SEG_ITER is read into host memory");
      TV_CK(cudaStreamSynchronize(st->stream));
      *static_cast<int*>(dst) = st->iter;
      return SHF_OK;
    }
    default: return tv_fail(SHF_ERR_ARG, "tv_admm_get: unknown selector");
  }
}

int tv_admm_set(tv_state* st, int what, const void* src, int on_host) {
  if (!st || !src) return tv_fail(SHF_ERR_ARG, "tv_admm_set: NULL argument");
  const size_t P = st->P(), K = st->K;
  const cudaMemcpyKind kind = on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  int rc = SHF_OK;
  switch (what) {
    case SEG_W: rc = tv_copy(st, st->w, src, sizeof(float) * P * K, kind, false); break;
    case SEG_BW: rc = tv_copy(st, st->bw, src, sizeof(float) * P * K, kind, false); break;
    case SEG_BV: rc = tv_copy(st, st->bv, src, sizeof(float) * 2 * P * K, kind, false); break;
    case SEG_V: {  // d = v - b_v with the current b_v
      rc = tv_copy(st, st->d, src, sizeof(float) * 2 * P * K, kind, false);
      if (rc == SHF_OK) {
        k_axpb<<<grid_for(2 * P * K), kThreads, 0, st->stream>>>(st->d, st->bv, st->d, -1.f, 2 * P * K);
        TV_CK(cudaGetLastError());
      }
      break;
    }
    default: return tv_fail(SHF_ERR_ARG, "tv_admm_set: accepts SEG_W, SEG_BW, SEG_BV and SEG_V");
  }
  if (rc) return rc;
  TV_CK(rebuild_rhs(st));
  TV_CK(cudaStreamSynchronize(st->stream));
  return SHF_OK;
}

int tv_admm_sync(tv_state* st) {
  if (!st) return tv_fail(SHF_ERR_ARG, "tv_admm_sync: NULL state");
  TV_CK(cudaStreamSynchronize(st->stream));
  return SHF_OK;
}

int tv_admm_destroy(tv_state* st) {
  free_tv(st);
  return SHF_OK;
}

}  // extern "C"

// Reverse mode of the unrolled ADMM of Sec. 3 (Haeuser & Steidl,
// arXiv:1112.1805): the per-pixel and per-coefficient parts of the adjoint of
// one iteration.  The transforms of the adjoint are the forward ones with the
// roles of S and S^T exchanged (the frame is Parseval, S^T is the adjoint).
//
// One iteration maps (b_v, Q = S^T(v - b_v), w, b_w) to
//   u = (Q + w - b_w - gamma s)/2, g = b_v + S u, b_v' = clip(g, t_f),
//   Q' = S^T(g - 2 clip(g, t_f)), g_w = b_w + u, w' = P_C(g_w), b_w' = g_w - w';
// its adjoint, given the adjoints of the outputs, is
//   gbar_w = bwbar' + J_P(wbar' - bwbar'),  dbar = S Qbar',
//   gbar = dbar (1 - 2 m) + bvbar' m,  tbar_f += sum sign(g)(1 - m)(bvbar' - 2 dbar),
//   ubar = gbar_w + S^T gbar,  Qbar = wbar = ubar/2,  bwbar = gbar_w - ubar/2,
//   bvbar = gbar,  sbar += -gamma ubar/2,
// with m = [|g| < t_f] and J_P the Jacobian of the simplex projection.
#include "shf_internal.h"

namespace shf {

namespace {

constexpr int kThreads = 256;
constexpr int kPartBlocks = 256;

// J_P x = x_A - mean_A(x) on the support A of the projection, 0 elsewhere.
__global__ void k_adj_proj(const float* __restrict__ wn, const float* __restrict__ wbar,
                           const float* __restrict__ bwbar, float* __restrict__ gwbar, int K, int P) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < P; r += gridDim.x * blockDim.x) {
    int q = 0;
    float mean = 0.f;
    for (int k = 0; k < K; ++k) {
      const size_t i = static_cast<size_t>(k) * P + r;
      if (wn[i] > 0.f) {
        ++q;
        mean += wbar[i] - bwbar[i];
      }
    }
    mean = q > 0 ? mean / static_cast<float>(q) : 0.f;
    for (int k = 0; k < K; ++k) {
      const size_t i = static_cast<size_t>(k) * P + r;
      const float a = wbar[i] - bwbar[i];
      gwbar[i] = bwbar[i] + (wn[i] > 0.f ? a - mean : 0.f);
    }
  }
}

__device__ double block_sum(double v) {
  __shared__ double buf[kThreads];
  buf[threadIdx.x] = v;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) buf[threadIdx.x] += buf[threadIdx.x + s];
    __syncthreads();
  }
  const double r = buf[0];
  __syncthreads();
  return r;
}

// grid (kPartBlocks, planes); plane = k * eta + f.
__global__ void __launch_bounds__(kThreads)
    k_adj_shrink(const float* __restrict__ g, const float* __restrict__ dbar, float* __restrict__ bvbar,
                 const float* __restrict__ thr, int eta, long P, double* __restrict__ tpart) {
  const size_t plane = blockIdx.y;
  const float t = thr[plane % eta];
  const size_t base = plane * static_cast<size_t>(P);
  float acc = 0.f;  // per thread in FP32 (fixed order), across the block in FP64
  for (long r = blockIdx.x * static_cast<long>(kThreads) + threadIdx.x; r < P;
       r += static_cast<long>(gridDim.x) * kThreads) {
    const float gv = g[base + r], db = dbar[base + r], bb = bvbar[base + r];
    if (fabsf(gv) < t) {
      bvbar[base + r] = bb - db;
    } else {
      bvbar[base + r] = db;
      acc = fmaf(gv > 0.f ? 1.f : -1.f, fmaf(-2.f, db, bb), acc);
    }
  }
  const double s = block_sum(static_cast<double>(acc));
  if (threadIdx.x == 0) tpart[plane * gridDim.x + blockIdx.x] = s;
}

// tbar[f] += sum over labels k and parts j < n of tpart[(k eta + f) n + j]:
// one block per filter; thread t sums the parts j = t, t + kThreads, ... of
// every label in order, then a fixed tree (deterministic).
__global__ void __launch_bounds__(kThreads) k_adj_tsum(const double* __restrict__ tpart, int K, int eta, int n,
                                                       double* __restrict__ tbar) {
  const int f = blockIdx.x;
  double acc = 0.0;
  for (int k = 0; k < K; ++k) {
    const double* p = tpart + (static_cast<size_t>(k) * eta + f) * n;
    for (int j = threadIdx.x; j < n; j += kThreads) acc += p[j];
  }
  const double s = block_sum(acc);
  if (threadIdx.x == 0) tbar[f] += s;
}

__global__ void k_adj_u(const float* __restrict__ gwbar, const float* __restrict__ st, float* __restrict__ Qbar,
                        float* __restrict__ wbar, float* __restrict__ bwbar, float* __restrict__ sbar, float gamma,
                        long n) {
  for (long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long>(gridDim.x) * blockDim.x) {
    const float ub = gwbar[i] + st[i];
    Qbar[i] = 0.5f * ub;
    wbar[i] = 0.5f * ub;
    bwbar[i] = gwbar[i] - 0.5f * ub;
    sbar[i] += -0.5f * gamma * ub;
  }
}

struct Cb {
  float c[kMaxK * kMaxC];
};

// part[(k * C + ch) * kPartBlocks + blk] = block sums of sbar_k (-2)(f_ch - c_k,ch)
__global__ void __launch_bounds__(kThreads)
    k_adj_cb_part(const float* __restrict__ sbar, const float* __restrict__ f, Cb cb, int K, int C, long P,
                  double* __restrict__ part) {
  const int kc = blockIdx.y, k = kc / C, ch = kc % C;
  double acc = 0.0;
  for (long r = blockIdx.x * static_cast<long>(kThreads) + threadIdx.x; r < P;
       r += static_cast<long>(gridDim.x) * kThreads)
    acc += static_cast<double>(sbar[static_cast<size_t>(k) * P + r]) * -2.0 *
           (static_cast<double>(f[static_cast<size_t>(ch) * P + r]) - cb.c[k * C + ch]);
  const double s = block_sum(acc);
  if (threadIdx.x == 0) part[static_cast<size_t>(kc) * gridDim.x + blockIdx.x] = s;
}

__global__ void k_adj_cb_sum(const double* __restrict__ part, int n, int nblk, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double acc = 0.0;
  for (int b = 0; b < nblk; ++b) acc += part[static_cast<size_t>(i) * nblk + b];
  out[i] = acc;
}

__global__ void k_adj_fgrad(const float* __restrict__ sbar, const float* __restrict__ f, Cb cb, int K, int C, long P,
                            float* __restrict__ fbar) {
  for (long r = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; r < P;
       r += static_cast<long>(gridDim.x) * blockDim.x)
    for (int ch = 0; ch < C; ++ch) {
      float acc = 0.f;
      for (int k = 0; k < K; ++k)
        acc += sbar[static_cast<size_t>(k) * P + r] * 2.f * (f[static_cast<size_t>(ch) * P + r] - cb.c[k * C + ch]);
      fbar[static_cast<size_t>(ch) * P + r] = acc;
    }
}

int grid_for(long n) {
  long g = (n + kThreads - 1) / kThreads;
  return static_cast<int>(g < 1 ? 1 : (g > 4096 ? 4096 : g));
}

}  // namespace

int adj_part_blocks() { return kPartBlocks; }

cudaError_t launch_adj_proj(const float* wn, const float* wbar, const float* bwbar, float* gwbar, int K, int P,
                            cudaStream_t st) {
  k_adj_proj<<<grid_for(P), kThreads, 0, st>>>(wn, wbar, bwbar, gwbar, K, P);
  return cudaGetLastError();
}

cudaError_t launch_adj_shrink(const float* g, const float* dbar, float* bvbar, const float* thr, int K, int eta,
                              long P, double* tpart, double* tbar, cudaStream_t st) {
  k_adj_shrink<<<dim3(kPartBlocks, K * eta), kThreads, 0, st>>>(g, dbar, bvbar, thr, eta, P, tpart);
  k_adj_tsum<<<eta, kThreads, 0, st>>>(tpart, K, eta, kPartBlocks, tbar);
  return cudaGetLastError();
}

cudaError_t launch_adj_tsum_rows(const double* tpart, int K, int eta, int H, double* tbar, cudaStream_t st) {
  k_adj_tsum<<<eta, kThreads, 0, st>>>(tpart, K, eta, H, tbar);
  return cudaGetLastError();
}

cudaError_t launch_adj_u(const float* gwbar, const float* st_, float* Qbar, float* wbar, float* bwbar, float* sbar,
                         float gamma, long n, cudaStream_t st) {
  k_adj_u<<<grid_for(n), kThreads, 0, st>>>(gwbar, st_, Qbar, wbar, bwbar, sbar, gamma, n);
  return cudaGetLastError();
}

cudaError_t adj_codebook(const float* sbar, const float* f, const float* codebook_host, int K, int C, long P,
                         double* part, double* out_dev, float* fbar, cudaStream_t st) {
  Cb cb{};
  for (int i = 0; i < K * C; ++i) cb.c[i] = codebook_host[i];
  k_adj_cb_part<<<dim3(kPartBlocks, K * C), kThreads, 0, st>>>(sbar, f, cb, K, C, P, part);
  k_adj_cb_sum<<<1, 64, 0, st>>>(part, K * C, kPartBlocks, out_dev);
  if (fbar) k_adj_fgrad<<<grid_for(P), kThreads, 0, st>>>(sbar, f, cb, K, C, P, fbar);
  return cudaGetLastError();
}

}  // namespace shf

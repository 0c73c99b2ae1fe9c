// NL-means-regularised segmentation, the second comparison model of Sec. 4:
// the gradient of the TV model replaced by a matrix D built from patch
// similarities of the image f.
//
// Graph (once per image): the patch distance d_a(i, j) = sum over the p x p
// patch of G_a(t) sum_ch (f(i + t) - f(j + t))^2 (G_a the Gaussian of
// standard deviation a normalised to sum 1, f mirrored at the border) for
// every candidate j of the varpi x varpi search window (clipped to the image)
// is computed on the GPU in FP64 with every product and sum rounded
// separately, and each pixel's candidates are ranked by (distance, raster
// index).  The selection itself is sequential in the paper (pixels in
// raster order pick min(mt, 2 mt - l) new neighbours, l the neighbours they
// already have, and links are symmetric), so it runs on the host over the
// ranked lists; a candidate already linked or holding 2 mt neighbours is
// passed over.
//
// ADMM (Sec. 3 with S replaced by D, per iteration):
//   u   = (I + D^T D)^(-1) [ D^T (v - b_v) + (w - b_w) - gamma s ]
//   v   = group shrinkage of g = b_v + D u over the m K values of a pixel,
//         b_v = g - v (kept as b_v and d = v - b_v)
//   w   = simplex projection of b_w + u, b_w = b_w + u - w.
// D^T D = 2 L (L the graph Laplacian of the symmetric neighbour sets), so
// I + D^T D has its spectrum in [1, 1 + 4 deg_max]; the u-step runs a fixed
// number of Chebyshev iterations on that interval from the previous u (no
// inner products, one launch per step), enough for a relative error below
// 1e-7 of the initial one.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "shearseg.h"
#include "shf_fast.h"
#include "shf_internal.h"
#include "shf_simplex.cuh"

struct nl_state {
  int H = 0, W = 0, K = 0, C = 0, m = 0, device = 0, deg_max = 0;
  float gamma = 1.f, lambda = 0.f;
  nl_params prm{};
  std::vector<float> codebook;
  std::vector<int> nbr_host, deg_host;  // [P][m] (increasing index, -1 padded), [P]
  std::vector<float> cheb_a, cheb_c;    // Chebyshev coefficients per step
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  float *f = nullptr, *s = nullptr, *u = nullptr, *bv = nullptr, *d = nullptr;
  float *w = nullptr, *bw = nullptr, *q = nullptr, *gap = nullptr;
  // the u-step's vectors pixel-major, four labels per float4 ([P][Q], Q = ceil(K/4)):
  // two Chebyshev iterates, the Chebyshev direction and the right-hand side
  float4 *xa = nullptr, *xb = nullptr, *cd = nullptr, *rhs = nullptr;
  int Q = 0;
  int* nbr = nullptr;                   // [m][P]
  short* off = nullptr;                 // [m][P] neighbour minus pixel index (|off| <= 7 W + 7)
  unsigned char *rev = nullptr, *deg = nullptr;
  int* labels = nullptr;
  int* flag = nullptr;
  double* red = nullptr;
  // the persistent Chebyshev solve (K <= 4 and the image within one resident
  // grid): its barrier counter and timeout flag, the steps' (a, c), its grid
  unsigned* cbar = nullptr;
  int* cerr = nullptr;
  float2* cheb_ac = nullptr;
  int cheb_grid = 0, cheb_halo = 0;
  int iter = 0;
  cudaGraphExec_t exec = nullptr;
  bool graph_tried = false;
  size_t P() const { return static_cast<size_t>(H) * W; }
};

namespace {

constexpr int kThreads = 256;
constexpr int kRedBlocks = 512;
constexpr int kMaxM = 16;       // neighbours per pixel (2 mt, mt <= 8)
constexpr int kMaxWin = 15;     // search window side: (2r + 1)^2 <= 225 window codes
constexpr int kMaxPatch = 9;    // patch side
constexpr int kRankWarps = 4;   // warps (pixels) per CTA of the ranking kernel

__device__ __forceinline__ int mirror_idx(int x, int n) {
  while (x < 0 || x >= n) x = x < 0 ? -x : 2 * (n - 1) - x;
  return x;
}

// One warp per pixel: the patch distances to every window code c = (dy + r)
// (2r + 1) + (dx + r) (the centre and codes outside the image excluded) and
// their ranks by (distance, code); rank[i][pos] = code of position pos, 255
// for the unused positions at the end.  Codes in increasing order are
// candidates in increasing raster index, so this is the order (distance,
// raster index).  G: the patch weights [(2h+1)^2] in FP64.
__global__ void __launch_bounds__(32 * kRankWarps) k_nl_rank(const float* __restrict__ f, int H, int W, int C,
                                                             const double* __restrict__ G, int h, int r,
                                                             unsigned char* __restrict__ rank) {
  __shared__ double key[kRankWarps][(2 * (kMaxWin / 2) + 1) * (2 * (kMaxWin / 2) + 1)];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int i = blockIdx.x * kRankWarps + wid;
  const int side = 2 * r + 1, NW = side * side;
  const size_t P = static_cast<size_t>(H) * W;
  if (i >= H * W) return;  // whole warps leave together
  const int ri = i / W, ci = i - ri * W;
  const int n = 2 * h + 1;
  for (int c = lane; c < NW; c += 32) {
    const int dy = c / side - r, dx = c % side - r;
    const int rj = ri + dy, cj = ci + dx;
    double acc = INFINITY;
    if ((dy != 0 || dx != 0) && rj >= 0 && rj < H && cj >= 0 && cj < W) {
      acc = 0.0;
      for (int t1 = -h; t1 <= h; ++t1)
        for (int t2 = -h; t2 <= h; ++t2) {
          const size_t a = static_cast<size_t>(mirror_idx(ri + t1, H)) * W + mirror_idx(ci + t2, W);
          const size_t b = static_cast<size_t>(mirror_idx(rj + t1, H)) * W + mirror_idx(cj + t2, W);
          double sum = 0.0;
          for (int ch = 0; ch < C; ++ch) {
            const double dd = __dsub_rn(static_cast<double>(f[ch * P + a]), static_cast<double>(f[ch * P + b]));
            sum = __dadd_rn(sum, __dmul_rn(dd, dd));
          }
          acc = __dadd_rn(acc, __dmul_rn(G[(t1 + h) * n + (t2 + h)], sum));
        }
    }
    key[wid][c] = acc;
  }
  __syncwarp();
  unsigned char* out = rank + static_cast<size_t>(i) * NW;
  for (int c = lane; c < NW; c += 32) {
    const double kc = key[wid][c];
    int pos = 0;
    for (int c2 = 0; c2 < NW; ++c2) {
      const double k2 = key[wid][c2];
      pos += (k2 < kc || (k2 == kc && c2 < c)) ? 1 : 0;
    }
    out[pos] = kc == INFINITY ? 255 : static_cast<unsigned char>(c);
  }
}

// The neighbours of pixel i into registers: nb[b] for b < deg(i).
__device__ __forceinline__ int load_nbrs(const int* __restrict__ nbr, const unsigned char* __restrict__ deg, size_t P,
                                         size_t i, int m, int (&nb)[kMaxM]) {
  const int dg = deg[i];
#pragma unroll
  for (int b = 0; b < kMaxM; ++b) nb[b] = (b < dg && b < m) ? nbr[b * P + i] : 0;
  return dg;
}

// One Chebyshev step for (I + D^T D) x = rhs on every label:
// r = rhs - x - 2 (deg x - sum_nbrs x), d <- a d + c r, x_out = x_in + d.
// The iterates, the direction and the right-hand side are pixel-major, four
// labels per float4, so that each neighbour is one 16-byte load per four
// labels; the first step reads u label-major ([K][P], IN_LM) and the last
// writes it back label-major (OUT_LM).
__device__ __forceinline__ float4 f4_axpy(float a, float4 x, float4 y) {
  return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}

template <bool IN_LM, bool OUT_LM>
__global__ void __launch_bounds__(kThreads) k_nl_cheb(const float* __restrict__ xin_lm, const float4* __restrict__ xin,
                                                      float* __restrict__ xout_lm, float4* __restrict__ xout,
                                                      float4* __restrict__ d, const float4* __restrict__ rhs,
                                                      const short* __restrict__ off,
                                                      const unsigned char* __restrict__ deg, int K, int Q, int m,
                                                      size_t P, float a, float c) {
  shf::fast::pdl_wait();  // x and d come from the previous step
  shf::fast::pdl_trigger();
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < P;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const int dg = deg[i];
    int nb[kMaxM];
#pragma unroll
    for (int b = 0; b < kMaxM; ++b) nb[b] = (b < dg && b < m) ? static_cast<int>(i) + off[b * P + i] : 0;
    auto load = [&](size_t j, int qd) -> float4 {
      if constexpr (IN_LM) {
        const int k0 = 4 * qd;
        return make_float4(xin_lm[k0 * P + j], k0 + 1 < K ? xin_lm[(k0 + 1) * P + j] : 0.f,
                           k0 + 2 < K ? xin_lm[(k0 + 2) * P + j] : 0.f, k0 + 3 < K ? xin_lm[(k0 + 3) * P + j] : 0.f);
      } else {
        return xin[j * Q + qd];
      }
    };
    for (int qd = 0; qd < Q; ++qd) {
      const float4 xi = load(i, qd);
      float4 sn = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int b = 0; b < kMaxM; ++b) {
        if (b < dg) {
          const float4 xn = load(static_cast<size_t>(nb[b]), qd);
          sn = make_float4(sn.x + xn.x, sn.y + xn.y, sn.z + xn.z, sn.w + xn.w);
        }
      }
      const float fd = static_cast<float>(dg);
      const float4 rh = rhs[i * Q + qd];
      const float4 res = make_float4(rh.x - (xi.x + 2.f * (fd * xi.x - sn.x)), rh.y - (xi.y + 2.f * (fd * xi.y - sn.y)),
                                     rh.z - (xi.z + 2.f * (fd * xi.z - sn.z)), rh.w - (xi.w + 2.f * (fd * xi.w - sn.w)));
      const float4 dn = f4_axpy(c, res, make_float4(a * d[i * Q + qd].x, a * d[i * Q + qd].y, a * d[i * Q + qd].z,
                                                     a * d[i * Q + qd].w));
      d[i * Q + qd] = dn;
      const float4 xo = make_float4(xi.x + dn.x, xi.y + dn.y, xi.z + dn.z, xi.w + dn.w);
      if constexpr (OUT_LM) {
        const int k0 = 4 * qd;
        xout_lm[k0 * P + i] = xo.x;
        if (k0 + 1 < K) xout_lm[(k0 + 1) * P + i] = xo.y;
        if (k0 + 2 < K) xout_lm[(k0 + 2) * P + i] = xo.z;
        if (k0 + 3 < K) xout_lm[(k0 + 3) * P + i] = xo.w;
      } else {
        xout[i * Q + qd] = xo;
      }
    }
  }
}

// The whole Chebyshev solve in one cooperative launch (K <= 4: one float4 per
// pixel), for images whose pixels fit the resident grid.  CTA c owns the
// contiguous pixels [c B, c B + B), B = kChebThreads kChebPPT; each thread
// keeps its pixels' right-hand side, direction d and iterate in registers for
// all the steps, and the CTA keeps its pixels' neighbour offsets (at most MM
// per pixel) in shared memory.  Per step the CTA copies the iterate on the
// window halo of its pixels (R = r W + r pixels on each side: every neighbour
// offset falls inside it) from the previous step's buffer into shared memory
// (asynchronous copies through L2), puts its own pixels there from registers,
// gathers the neighbours there, and writes its pixels to the other buffer; a
// grid barrier separates the steps.  The arithmetic is k_nl_cheb's, in its
// order.
constexpr int kChebPPT = 2;
constexpr int kChebThreads = 1024;
constexpr int kChebBlock = kChebPPT * kChebThreads;         // pixels per CTA
constexpr unsigned long long kBarrierNs = 1000000000ull;  // a barrier gives up after one second

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned load_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier number gen (1, 2, ...) on a counter that was zero at launch:
// every CTA adds one and waits until gen * gridDim.x CTAs have arrived.  The
// wait is bounded: after kBarrierNs it sets *err and the barrier reports
// failure (every CTA then leaves the kernel; the host reads *err).
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned gen, int* err) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    // release: the CTA's writes (ordered before this thread by the CTA
    // barrier) become visible with the arrival; acquire on the way out
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
    const unsigned target = gen * gridDim.x;
    const unsigned long long t0 = global_ns();
    int ok = 1;
    while (load_acquire(bar) < target) {
      if (global_ns() - t0 > kBarrierNs) {
        ok = 0;
        atomicExch(err, 1);
        break;
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

template <int MM>
__global__ void __launch_bounds__(kChebThreads, 1) k_nl_cheb_all(float* __restrict__ u, float4* xa, float4* xb,
                                                               const float4* __restrict__ rhs,
                                                               const short* __restrict__ off,
                                                               const unsigned char* __restrict__ deg, int K, int m,
                                                               size_t P, int R, int nsteps,
                                                               const float2* __restrict__ ac, unsigned* bar,
                                                               int* err) {
  extern __shared__ __align__(16) float4 sx[];  // the iterate on [lo, hi), then the offsets
  short* so = reinterpret_cast<short*>(sx + kChebBlock + 2 * static_cast<size_t>(R));  // [MM][kChebBlock]
  const size_t base = static_cast<size_t>(blockIdx.x) * kChebBlock;
  const size_t lo = base > static_cast<size_t>(R) ? base - R : 0;
  const size_t hi = base + kChebBlock + R < P ? base + kChebBlock + R : P;
  for (int e = threadIdx.x; e < MM * kChebBlock; e += kChebThreads) {
    const int b = e / kChebBlock, j = e - b * kChebBlock;
    const size_t i = base + j;
    so[e] = (i < P && b < m) ? off[b * P + i] : static_cast<short>(0);
  }
  int dg[kChebPPT];
  float4 r[kChebPPT], dd[kChebPPT], xi[kChebPPT];
#pragma unroll
  for (int p = 0; p < kChebPPT; ++p) {
    const size_t i = base + p * kChebThreads + threadIdx.x;
    const bool live = i < P;
    dg[p] = live ? min(static_cast<int>(deg[i]), m) : 0;
    r[p] = live ? rhs[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    dd[p] = make_float4(0.f, 0.f, 0.f, 0.f);
    xi[p] = live ? make_float4(u[i], K > 1 ? u[P + i] : 0.f, K > 2 ? u[2 * P + i] : 0.f, K > 3 ? u[3 * P + i] : 0.f)
                 : make_float4(0.f, 0.f, 0.f, 0.f);
    if (live) xa[i] = xi[p];
  }
  if (!grid_barrier(bar, 1, err)) return;
  const float4* xin = xa;
  float4* xout = xb;
  for (int k = 0; k < nsteps; ++k) {
    // the halos by asynchronous 16-byte copies (through L2: other CTAs wrote
    // them in the previous step), all in flight at once; the CTA's own
    // pixels from registers
    const size_t own_end = base + kChebBlock < hi ? base + kChebBlock : hi;
    for (size_t j = lo + threadIdx.x; j < hi; j += kChebThreads) {
      if (j >= base && j < own_end) continue;
      const unsigned dst = static_cast<unsigned>(__cvta_generic_to_shared(sx + (j - lo)));
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(xin + j) : "memory");
    }
#pragma unroll
    for (int p = 0; p < kChebPPT; ++p) {
      const size_t i = base + p * kChebThreads + threadIdx.x;
      if (i < P) sx[i - lo] = xi[p];
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    const float a = ac[k].x, c = ac[k].y;
#pragma unroll
    for (int p = 0; p < kChebPPT; ++p) {
      const size_t i = base + p * kChebThreads + threadIdx.x;
      if (i >= P) continue;
      const long long il = static_cast<long long>(i - lo);
      const short* sop = so + p * kChebThreads + threadIdx.x;
      float4 sn = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int b = 0; b < MM; ++b) {
        if (b < dg[p]) {
          const float4 xn = sx[il + sop[b * kChebBlock]];
          sn = make_float4(sn.x + xn.x, sn.y + xn.y, sn.z + xn.z, sn.w + xn.w);
        }
      }
      const float fd = static_cast<float>(dg[p]);
      const float4 x = xi[p], rh = r[p], d0 = dd[p];
      const float4 res = make_float4(rh.x - (x.x + 2.f * (fd * x.x - sn.x)), rh.y - (x.y + 2.f * (fd * x.y - sn.y)),
                                     rh.z - (x.z + 2.f * (fd * x.z - sn.z)), rh.w - (x.w + 2.f * (fd * x.w - sn.w)));
      const float4 dn = f4_axpy(c, res, make_float4(a * d0.x, a * d0.y, a * d0.z, a * d0.w));
      dd[p] = dn;
      xi[p] = make_float4(x.x + dn.x, x.y + dn.y, x.z + dn.z, x.w + dn.w);
      if (k + 1 < nsteps) xout[i] = xi[p];
    }
    if (k + 1 < nsteps) {
      if (!grid_barrier(bar, static_cast<unsigned>(k) + 2u, err)) return;  // also orders the shared reads
      const float4* t = xout;
      xout = const_cast<float4*>(xin);
      xin = t;
    }
  }
#pragma unroll
  for (int p = 0; p < kChebPPT; ++p) {
    const size_t i = base + p * kChebThreads + threadIdx.x;
    if (i >= P) continue;
    u[i] = xi[p].x;
    if (K > 1) u[P + i] = xi[p].y;
    if (K > 2) u[2 * P + i] = xi[p].z;
    if (K > 3) u[3 * P + i] = xi[p].w;
  }
}

// The barrier with a target no CTA reaches (each arrives once, generation 2
// needs two arrivals each): the bounded wait must give up (self-test).
__global__ void k_barrier_unreachable(unsigned* bar, int* err) { grid_barrier(bar, 2, err); }

// Shared memory of the persistent solve: the iterate on the CTA's pixels and
// two halos, and MM neighbour offsets per pixel.
size_t cheb_all_smem(int R, int MM) {
  return sizeof(float4) * (static_cast<size_t>(kChebBlock) + 2 * static_cast<size_t>(R)) +
         sizeof(short) * static_cast<size_t>(MM) * kChebBlock;
}

// The v-, w- and b-updates after the u-step: g_b = b_v,b + u(nbr_b) - u(i)
// (b < deg; b_v,b for the zero rows), group clip over the m K values,
// d = g - 2 b_v; w-step and q = (w - b_w) - gamma s.
template <int KM>
__global__ void __launch_bounds__(kThreads) k_nl_prox(const float* __restrict__ u, float* __restrict__ bv,
                                                      float* __restrict__ d, float* __restrict__ w,
                                                      float* __restrict__ bw, const float* __restrict__ s,
                                                      float* __restrict__ q, const int* __restrict__ nbr,
                                                      const unsigned char* __restrict__ deg, int K, int m, size_t P,
                                                      float t, float gamma) {
  shf::fast::pdl_wait();  // u comes from the last Chebyshev step
  shf::fast::pdl_trigger();
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < P;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    int nb[kMaxM];
    const int dg = load_nbrs(nbr, deg, P, i, m, nb);
    // the group norm over the m K values of g (the label loop is not unrolled:
    // only the neighbour indices stay in registers)
    float n2 = 0.f;
    for (int k = 0; k < K; ++k) {
      const float* up = u + k * P;
      const float ui = up[i];
      const float* bk = bv + static_cast<size_t>(k) * m * P;
#pragma unroll
      for (int b = 0; b < kMaxM; ++b) {
        if (b < m) {
          const float g = bk[b * P + i] + (b < dg ? up[nb[b]] - ui : 0.f);
          n2 = fmaf(g, g, n2);
        }
      }
    }
    const float nrm = sqrtf(n2);
    const float fac = nrm > t ? t / nrm : 1.f;
    for (int k = 0; k < K; ++k) {
      const float* up = u + k * P;
      const float ui = up[i];
      float* bk = bv + static_cast<size_t>(k) * m * P;
      float* dk = d + static_cast<size_t>(k) * m * P;
#pragma unroll
      for (int b = 0; b < kMaxM; ++b) {
        if (b < m) {
          const float g = bk[b * P + i] + (b < dg ? up[nb[b]] - ui : 0.f);
          const float bn = fac * g;
          bk[b * P + i] = bn;
          dk[b * P + i] = g - 2.f * bn;
        }
      }
    }
    float gw[KM], wk[KM];
#pragma unroll
    for (int k = 0; k < KM; ++k) {
      gw[k] = k < K ? bw[k * P + i] + u[k * P + i] : 0.f;
      wk[k] = gw[k];
    }
    shf::simplex_project<KM>(wk, K);
#pragma unroll
    for (int k = 0; k < KM; ++k) {
      if (k < K) {
        const float bn = gw[k] - wk[k];
        w[k * P + i] = wk[k];
        bw[k * P + i] = bn;
        q[k * P + i] = (wk[k] - bn) - gamma * s[k * P + i];
      }
    }
  }
}

// rhs = q + D^T d: (D^T d)(j) = sum_{b < deg(j)} [d_rev(j,b)(nbr_b(j)) - d_b(j)],
// written pixel-major ([P][4 Q], labels K..4Q-1 zero) for the Chebyshev steps.
__global__ void __launch_bounds__(kThreads) k_nl_rhs(const float* __restrict__ q, const float* __restrict__ d,
                                                     float* __restrict__ rhs, const int* __restrict__ nbr,
                                                     const unsigned char* __restrict__ rev,
                                                     const unsigned char* __restrict__ deg, int K, int Q, int m,
                                                     size_t P) {
  shf::fast::pdl_wait();  // q and d come from the prox kernel
  shf::fast::pdl_trigger();
  for (size_t j = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; j < P;
       j += static_cast<size_t>(gridDim.x) * blockDim.x) {
    int nb[kMaxM];
    const int dg = load_nbrs(nbr, deg, P, j, m, nb);
    int rv[kMaxM];
#pragma unroll
    for (int b = 0; b < kMaxM; ++b) rv[b] = b < dg ? rev[b * P + j] : 0;
    for (int k = 0; k < K; ++k) {
      const float* dk = d + static_cast<size_t>(k) * m * P;
      float acc = 0.f;
#pragma unroll
      for (int b = 0; b < kMaxM; ++b)
        if (b < dg) acc += dk[rv[b] * P + nb[b]] - dk[b * P + j];
      rhs[j * 4 * Q + k] = q[k * P + j] + acc;  // pixel-major, four labels per float4
    }
    for (int k = K; k < 4 * Q; ++k) rhs[j * 4 * Q + k] = 0.f;
  }
}

__global__ void k_nl_q(const float* __restrict__ w, const float* __restrict__ bw, const float* __restrict__ s,
                       float* __restrict__ q, float gamma, size_t n) {
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * blockDim.x)
    q[i] = (w[i] - bw[i]) - gamma * s[i];
}

// out = a + sb b (out may alias a).
__global__ void k_nl_axpb(const float* a, const float* __restrict__ b, float* out, float sb, size_t n) {
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * blockDim.x)
    out[i] = a[i] + sb * b[i];
}

// FP64 energy partials: <w, s> and sum_i (sum_k sum_b ((D w_k)_b(i))^2)^(1/2).
__global__ void __launch_bounds__(kThreads) k_nl_energy(const float* __restrict__ w, const float* __restrict__ s,
                                                        const int* __restrict__ nbr,
                                                        const unsigned char* __restrict__ deg, int K, int m, size_t P,
                                                        double* __restrict__ partial) {
  double ds = 0.0, dt = 0.0;
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < P;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    int nb[kMaxM];
    const int dg = load_nbrs(nbr, deg, P, i, m, nb);
    double n2 = 0.0;
    for (int k = 0; k < K; ++k) {
      const float* wp = w + k * P;
      ds += static_cast<double>(wp[i]) * s[k * P + i];
#pragma unroll
      for (int b = 0; b < kMaxM; ++b) {
        if (b < dg) {
          const double e = static_cast<double>(wp[nb[b]]) - wp[i];
          n2 += e * e;
        }
      }
    }
    dt += sqrt(n2);
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

__global__ void k_nl_energy_final(const double* __restrict__ partial, int nblocks, double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double a = 0.0, b = 0.0;
  for (int i = 0; i < nblocks; ++i) {
    a += partial[2 * i];
    b += partial[2 * i + 1];
  }
  out[0] = a;
  out[1] = b;
}

int nl_fail(int code, const std::string& msg) { return shf::set_error(code, msg); }

#define NL_CK(call)                                                                                         \
  do {                                                                                                      \
    cudaError_t e_ = (call);                                                                                \
    if (e_ != cudaSuccess) return nl_fail(SHF_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <typename T>
int nl_alloc(T** p, size_t count, const char* what) {
  *p = nullptr;
  if (count == 0) return SHF_OK;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return nl_fail(e == cudaErrorMemoryAllocation ? SHF_ERR_OOM : SHF_ERR_CUDA,
                   std::string("cudaMalloc(") + what + "): " + cudaGetErrorString(e));
  }
  return SHF_OK;
}

int grid_for(size_t n) {
  const size_t b = (n + kThreads - 1) / kThreads;
  return static_cast<int>(b < 8192 ? (b ? b : 1) : 8192);
}

void free_nl(nl_state* st) {
  if (!st) return;
  if (st->stream) cudaStreamSynchronize(st->stream);
  if (st->exec) cudaGraphExecDestroy(st->exec);
  void* bufs[] = {st->f, st->s, st->u, st->xa, st->xb, st->cd, st->bv, st->d, st->w, st->bw, st->q, st->rhs,
                  st->gap, st->nbr, st->off, st->rev, st->deg, st->labels, st->flag, st->red,
                  st->cbar, st->cerr, st->cheb_ac};
  for (void* b : bufs) cudaFree(b);
  if (st->own_stream && st->stream) cudaStreamDestroy(st->stream);
  delete st;
}

// Patch weights G_a on the (2h+1)^2 patch, normalised to sum 1.
std::vector<double> patch_weights(int h, double a) {
  const int n = 2 * h + 1;
  std::vector<double> G(static_cast<size_t>(n) * n);
  double sum = 0.0;
  for (int t1 = -h; t1 <= h; ++t1)
    for (int t2 = -h; t2 <= h; ++t2) {
      const double g = std::exp(-static_cast<double>(t1 * t1 + t2 * t2) / (2.0 * a * a));
      G[(t1 + h) * n + (t2 + h)] = g;
      sum += g;
    }
  for (double& g : G) g /= sum;
  return G;
}

// The graph of st->f: ranks on the GPU, the sequential selection here; then
// the device tables (neighbours [m][P], reverse positions, counts) and the
// Chebyshev coefficients.  Synchronises.
int build_graph(nl_state* st) {
  const int H = st->H, W = st->W, mt = st->prm.neighbours, m = st->m;
  const int h = st->prm.patch / 2, r = st->prm.window / 2, side = 2 * r + 1, NW = side * side;
  const size_t P = st->P();
  const auto G = patch_weights(h, st->prm.a);
  double* dG = nullptr;
  unsigned char* drank = nullptr;
  NL_CK(cudaMallocAsync(reinterpret_cast<void**>(&dG), sizeof(double) * G.size(), st->stream));
  NL_CK(cudaMallocAsync(reinterpret_cast<void**>(&drank), P * NW, st->stream));
  std::vector<unsigned char> rank(P * NW);
  cudaError_t e = cudaMemcpyAsync(dG, G.data(), sizeof(double) * G.size(), cudaMemcpyHostToDevice, st->stream);
  if (e == cudaSuccess) {
    k_nl_rank<<<static_cast<unsigned>((P + kRankWarps - 1) / kRankWarps), 32 * kRankWarps, 0, st->stream>>>(
        st->f, H, W, st->C, dG, h, r, drank);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(rank.data(), drank, P * NW, cudaMemcpyDeviceToHost, st->stream);
  cudaError_t e2 = cudaFreeAsync(dG, st->stream);
  cudaError_t e3 = cudaFreeAsync(drank, st->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st->stream);
  if (e == cudaSuccess) e = e2 != cudaSuccess ? e2 : e3;
  NL_CK(e);
  // selection in raster order over the ranked candidates
  std::vector<int>& nb = st->nbr_host;
  std::vector<int>& dg = st->deg_host;
  nb.assign(P * m, -1);
  dg.assign(P, 0);
  for (size_t i = 0; i < P; ++i) {
    const int ri = static_cast<int>(i / W), ci = static_cast<int>(i % W);
    const int k = std::min(mt, m - dg[i]);
    int taken = 0;
    for (int pos = 0; pos < NW && taken < k; ++pos) {
      const int c = rank[i * NW + pos];
      if (c == 255) break;  // the rest lie outside the image
      const int j = (ri + c / side - r) * W + (ci + c % side - r);
      if (dg[j] >= m) continue;
      bool linked = false;
      for (int b = 0; b < dg[i]; ++b) linked = linked || nb[i * m + b] == j;
      if (linked) continue;
      nb[i * m + dg[i]++] = j;
      nb[static_cast<size_t>(j) * m + dg[j]++] = static_cast<int>(i);
      ++taken;
    }
  }
  st->deg_max = 0;
  std::vector<int> nbt(P * m, -1);
  std::vector<unsigned char> rev(P * m, 0), deg8(P);
  for (size_t i = 0; i < P; ++i) {
    std::sort(nb.begin() + i * m, nb.begin() + i * m + dg[i]);
    st->deg_max = std::max(st->deg_max, dg[i]);
    deg8[i] = static_cast<unsigned char>(dg[i]);
    for (int b = 0; b < dg[i]; ++b) nbt[static_cast<size_t>(b) * P + i] = nb[i * m + b];
  }
  for (size_t i = 0; i < P; ++i)
    for (int b = 0; b < dg[i]; ++b) {  // position of i in the list of its b-th neighbour
      const int j = nb[i * m + b];
      int pos = 0;
      while (nb[static_cast<size_t>(j) * m + pos] != static_cast<int>(i)) ++pos;
      rev[static_cast<size_t>(b) * P + i] = static_cast<unsigned char>(pos);
    }
  std::vector<short> offs(P * m, 0);
  for (size_t e = 0; e < P * m; ++e)
    if (nbt[e] >= 0) offs[e] = static_cast<short>(nbt[e] - static_cast<long long>(e % P));
  NL_CK(cudaMemcpy(st->nbr, nbt.data(), sizeof(int) * P * m, cudaMemcpyHostToDevice));
  NL_CK(cudaMemcpy(st->off, offs.data(), sizeof(short) * P * m, cudaMemcpyHostToDevice));
  NL_CK(cudaMemcpy(st->rev, rev.data(), P * m, cudaMemcpyHostToDevice));
  NL_CK(cudaMemcpy(st->deg, deg8.data(), P, cudaMemcpyHostToDevice));
  // Chebyshev iteration on [1, 1 + 4 deg_max]: theta = centre, delta = half width
  const double lo = 1.0, hi = 1.0 + 4.0 * st->deg_max;
  const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo);
  int n = st->prm.solve_steps;
  if (n <= 0) {
    const double kappa = hi / lo;
    const double qrate = (std::sqrt(kappa) - 1.0) / (std::sqrt(kappa) + 1.0);
    n = qrate > 0.0 ? static_cast<int>(std::ceil(std::log(2.0 / 1e-7) / -std::log(qrate))) : 1;
  }
  n = std::max(n + (n & 1), 2);  // even and >= 2: the first step reads u, the last writes it
  st->cheb_a.assign(n, 0.f);
  st->cheb_c.assign(n, 0.f);
  st->cheb_c[0] = static_cast<float>(1.0 / theta);
  if (delta > 0.0) {
    const double sigma = theta / delta;
    double rho = 1.0 / sigma;
    for (int k = 1; k < n; ++k) {
      const double rn = 1.0 / (2.0 * sigma - rho);
      st->cheb_a[k] = static_cast<float>(rn * rho);
      st->cheb_c[k] = static_cast<float>(2.0 * rn / delta);
      rho = rn;
    }
  }
  // the persistent solve: the steps' (a, c) on the device, and its grid when
  // the pixels fit the resident CTAs at kChebPPT pixels per thread
  cudaFree(st->cheb_ac);
  st->cheb_ac = nullptr;
  st->cheb_grid = 0;
  // (the neighbours of a pixel lie in its window: |offset| <= r W + r)
  int coop = 0, sms = 0, per_sm = 0, optin = 0;
  st->cheb_halo = r * W + r;
  const int MM = m <= 10 ? 10 : kMaxM;
  const size_t smem = cheb_all_smem(st->cheb_halo, MM);
  const void* kern = MM == 10 ? reinterpret_cast<const void*>(k_nl_cheb_all<10>)
                              : reinterpret_cast<const void*>(k_nl_cheb_all<kMaxM>);
  if (st->Q == 1 && cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, st->device) == cudaSuccess && coop &&
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, st->device) == cudaSuccess &&
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, st->device) == cudaSuccess &&
      smem <= static_cast<size_t>(optin) &&
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) == cudaSuccess &&
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kChebThreads, smem) == cudaSuccess) {
    const size_t need = (P + kChebBlock - 1) / kChebBlock;
    if (need >= 1 && need <= static_cast<size_t>(per_sm) * sms) {
      std::vector<float2> ac(n);
      for (int k = 0; k < n; ++k) ac[k] = make_float2(st->cheb_a[k], st->cheb_c[k]);
      int rc = nl_alloc(&st->cheb_ac, static_cast<size_t>(n), "chebyshev coefficients");
      if (rc) return rc;
      NL_CK(cudaMemcpy(st->cheb_ac, ac.data(), sizeof(float2) * n, cudaMemcpyHostToDevice));
      st->cheb_grid = static_cast<int>(need);
    }
  }
  cudaGetLastError();
  return SHF_OK;
}

enum NlKind { kNlSolve = 0, kNlProx = 1, kNlRhs = 2, kNlKinds = 3 };
const char* const kNlNames[kNlKinds] = {"nl_solve", "nl_prox", "nl_rhs"};

cudaError_t launch_prox(nl_state* st) {
  const size_t P = st->P();
  const float t = st->gamma * st->lambda;
  const int grid = grid_for(P);
  if (st->K <= 4)
    return shf::fast::launch_pdl(k_nl_prox<4>, dim3(grid), dim3(kThreads), 0, st->stream, st->u, st->bv, st->d, st->w,
                                 st->bw, st->s, st->q, st->nbr, st->deg, st->K, st->m, P, t, st->gamma);
  else if (st->K <= 8)
    return shf::fast::launch_pdl(k_nl_prox<8>, dim3(grid), dim3(kThreads), 0, st->stream, st->u, st->bv, st->d, st->w,
                                 st->bw, st->s, st->q, st->nbr, st->deg, st->K, st->m, P, t, st->gamma);
  else
    return shf::fast::launch_pdl(k_nl_prox<16>, dim3(grid), dim3(kThreads), 0, st->stream, st->u, st->bv, st->d, st->w,
                                 st->bw, st->s, st->q, st->nbr, st->deg, st->K, st->m, P, t, st->gamma);
}

cudaError_t launch_rhs(nl_state* st) {
  return shf::fast::launch_pdl(k_nl_rhs, dim3(grid_for(st->P())), dim3(kThreads), 0, st->stream, st->q, st->d,
                               reinterpret_cast<float*>(st->rhs), st->nbr, st->rev, st->deg, st->K, st->Q, st->m,
                               st->P());
}

// One iteration; ev (nullable, kNlKinds + 1 events) recorded before each
// part and after the last.
cudaError_t enqueue_nl_iteration(nl_state* st, cudaEvent_t* ev) {
  cudaStream_t ss = st->stream;
  auto mark = [&](int i) { return ev ? cudaEventRecord(ev[i], ss) : cudaSuccess; };
  cudaError_t e = mark(kNlSolve);
  const size_t P = st->P();
  const int n = static_cast<int>(st->cheb_a.size());  // even, >= 2
  float4* x0 = st->xa;
  float4* x1 = st->xb;
  if (st->cheb_grid > 0 && e == cudaSuccess) {  // one cooperative launch for all the steps
    e = cudaMemsetAsync(st->cbar, 0, sizeof(unsigned), ss);
    if (e == cudaSuccess) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(st->cheb_grid);
      cfg.blockDim = dim3(kChebThreads);
      const int MM = st->m <= 10 ? 10 : kMaxM;
      cfg.dynamicSmemBytes = cheb_all_smem(st->cheb_halo, MM);
      cfg.stream = ss;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeCooperative;
      attr[0].val.cooperative = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      e = cudaLaunchKernelEx(&cfg, MM == 10 ? k_nl_cheb_all<10> : k_nl_cheb_all<kMaxM>, st->u, x0, x1, static_cast<const float4*>(st->rhs),
                             static_cast<const short*>(st->off), static_cast<const unsigned char*>(st->deg), st->K,
                             st->m, P, st->cheb_halo, n, static_cast<const float2*>(st->cheb_ac), st->cbar,
                             st->cerr);
    }
  }
  for (int k = 0; k < n && e == cudaSuccess && st->cheb_grid == 0; ++k) {
    const float a = st->cheb_a[k], c = st->cheb_c[k];
    const dim3 grid(grid_for(P)), block(kThreads);
    const float* none = nullptr;
    float* none_out = nullptr;
    const float4* none4 = nullptr;
    float4* none4_out = nullptr;
    if (k == 0)  // from u (label-major)
      e = shf::fast::launch_pdl(k_nl_cheb<true, false>, grid, block, 0, ss, st->u, none4, none_out, x0, st->cd,
                                st->rhs, st->off, st->deg, st->K, st->Q, st->m, P, a, c);
    else if (k == n - 1)  // back into u
      e = shf::fast::launch_pdl(k_nl_cheb<false, true>, grid, block, 0, ss, none, x0, st->u, none4_out, st->cd,
                                st->rhs, st->off, st->deg, st->K, st->Q, st->m, P, a, c);
    else {
      e = shf::fast::launch_pdl(k_nl_cheb<false, false>, grid, block, 0, ss, none, x0, none_out, x1, st->cd,
                                st->rhs, st->off, st->deg, st->K, st->Q, st->m, P, a, c);
      std::swap(x0, x1);
    }
  }
  if (e == cudaSuccess) e = mark(kNlProx);
  if (e == cudaSuccess) e = launch_prox(st);
  if (e == cudaSuccess) e = mark(kNlRhs);
  if (e == cudaSuccess) e = launch_rhs(st);
  if (e == cudaSuccess) e = mark(kNlKinds);
  return e;
}

cudaError_t rebuild_rhs(nl_state* st) {
  const size_t n = st->P() * st->K;
  k_nl_q<<<grid_for(n), kThreads, 0, st->stream>>>(st->w, st->bw, st->s, st->q, st->gamma, n);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? launch_rhs(st) : e;
}

// Graph, data term and the zero state.  Synchronises.
int nl_restart(nl_state* st) {
  const size_t P = st->P(), K = st->K, m = st->m;
  NL_CK(cudaMemsetAsync(st->flag, 0, sizeof(int), st->stream));
  NL_CK(shf::launch_count_nonfinite(st->f, static_cast<long>(P * st->C), st->flag, st->stream));
  int bad = 0;
  NL_CK(cudaMemcpyAsync(&bad, st->flag, sizeof(int), cudaMemcpyDeviceToHost, st->stream));
  NL_CK(cudaStreamSynchronize(st->stream));
  if (bad) return nl_fail(SHF_ERR_NONFINITE, "nl: the image contains NaN or Inf");
  int rc = build_graph(st);
  if (rc) return rc;
  if (st->exec) {  // the step count may have changed with the graph
    cudaGraphExecDestroy(st->exec);
    st->exec = nullptr;
    st->graph_tried = false;
  }
  NL_CK(shf::launch_data_term(st->f, st->C, st->codebook.data(), st->K, st->s, static_cast<int>(P), st->stream));
  NL_CK(cudaMemsetAsync(st->u, 0, sizeof(float) * P * K, st->stream));
  NL_CK(cudaMemsetAsync(st->w, 0, sizeof(float) * P * K, st->stream));
  NL_CK(cudaMemsetAsync(st->bw, 0, sizeof(float) * P * K, st->stream));
  NL_CK(cudaMemsetAsync(st->bv, 0, sizeof(float) * m * P * K, st->stream));
  NL_CK(cudaMemsetAsync(st->d, 0, sizeof(float) * m * P * K, st->stream));
  NL_CK(cudaMemsetAsync(st->cd, 0, sizeof(float4) * P * st->Q, st->stream));
  NL_CK(rebuild_rhs(st));
  NL_CK(cudaStreamSynchronize(st->stream));
  st->iter = 0;
  return SHF_OK;
}

int nl_copy(nl_state* st, void* dst, const void* src, size_t bytes, cudaMemcpyKind kind, bool sync) {
  NL_CK(cudaMemcpyAsync(dst, src, bytes, kind, st->stream));
  if (sync) NL_CK(cudaStreamSynchronize(st->stream));
  return SHF_OK;
}

}  // namespace

extern "C" {

int nl_admm_init(int H, int W, const float* f, int C, const float* codebook, int K, const nl_params* p, void* stream,
                 nl_state** out) {
  if (!out) return nl_fail(SHF_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!f || !codebook || !p) return nl_fail(SHF_ERR_ARG, "nl_admm_init: NULL argument");
  if (K < 2 || K > shf::kMaxK) return nl_fail(SHF_ERR_ARG, "K must be in [2, 16]");
  if (C != 1 && C != 3) return nl_fail(SHF_ERR_ARG, "C must be 1 or 3");
  if (!(p->gamma > 0.f) || !std::isfinite(p->gamma)) return nl_fail(SHF_ERR_ARG, "gamma must be positive and finite");
  if (!(p->lambda >= 0.f) || !std::isfinite(p->lambda))
    return nl_fail(SHF_ERR_ARG, "lambda must be finite and non-negative");
  if (p->patch < 1 || p->patch > kMaxPatch) return nl_fail(SHF_ERR_ARG, "patch must be in [1, 9]");
  if (p->window < 3 || p->window > kMaxWin || !(p->window & 1)) return nl_fail(SHF_ERR_ARG, "window must be odd, 3..15");
  if (!(p->a > 0.f) || !std::isfinite(p->a)) return nl_fail(SHF_ERR_ARG, "a must be positive");
  if (p->neighbours < 1 || 2 * p->neighbours > kMaxM) return nl_fail(SHF_ERR_ARG, "neighbours must be in [1, 8]");
  if (p->solve_steps < 0 || p->solve_steps > 1000) return nl_fail(SHF_ERR_ARG, "solve_steps must be in [0, 1000]");
  if (H < 8 || W < 8 || H > shf::kMaxSide || W > shf::kMaxSide) return nl_fail(SHF_ERR_SIZE, "H and W must be in [8, 2048]");
  if (reinterpret_cast<uintptr_t>(f) & 7u) return nl_fail(SHF_ERR_ARG, "f must be 8-byte aligned");
  for (int i = 0; i < K * C; ++i)
    if (!std::isfinite(codebook[i])) return nl_fail(SHF_ERR_NONFINITE, "codebook contains NaN or Inf");
  auto* st = new nl_state();
  st->H = H;
  st->W = W;
  st->K = K;
  st->C = C;
  st->prm = *p;
  st->m = 2 * p->neighbours;
  st->Q = (K + 3) / 4;
  st->gamma = p->gamma;
  st->lambda = p->lambda;
  st->codebook.assign(codebook, codebook + K * C);
  cudaError_t ed = cudaGetDevice(&st->device);
  if (ed != cudaSuccess) {
    delete st;
    return nl_fail(SHF_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(ed));
  }
  if (stream) {
    st->stream = static_cast<cudaStream_t>(stream);
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&st->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete st;
      return nl_fail(SHF_ERR_CUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
    }
    st->own_stream = true;
  }
  const size_t P = static_cast<size_t>(H) * W, m = st->m;
  int rc;
  if ((rc = nl_alloc(&st->f, P * C, "f")) || (rc = nl_alloc(&st->s, P * K, "s")) ||
      (rc = nl_alloc(&st->u, P * K, "u")) || (rc = nl_alloc(&st->xa, P * st->Q, "chebyshev x")) ||
      (rc = nl_alloc(&st->xb, P * st->Q, "chebyshev x")) || (rc = nl_alloc(&st->cd, P * st->Q, "chebyshev d")) ||
      (rc = nl_alloc(&st->bv, m * P * K, "b_v")) ||
      (rc = nl_alloc(&st->d, m * P * K, "d")) || (rc = nl_alloc(&st->w, P * K, "w")) ||
      (rc = nl_alloc(&st->bw, P * K, "b_w")) || (rc = nl_alloc(&st->q, P * K, "q")) ||
      (rc = nl_alloc(&st->rhs, P * st->Q, "rhs")) || (rc = nl_alloc(&st->gap, P, "gap")) ||
      (rc = nl_alloc(&st->nbr, P * m, "neighbours")) || (rc = nl_alloc(&st->off, P * m, "offsets")) ||
      (rc = nl_alloc(&st->rev, P * m, "reverse")) ||
      (rc = nl_alloc(&st->deg, P, "counts")) || (rc = nl_alloc(&st->labels, P, "labels")) ||
      (rc = nl_alloc(&st->flag, 1, "flag")) || (rc = nl_alloc(&st->red, 2 * kRedBlocks + 2, "red")) ||
      (rc = nl_alloc(&st->cbar, 1, "barrier")) || (rc = nl_alloc(&st->cerr, 1, "barrier flag"))) {
    free_nl(st);
    return rc;
  }
  if (cudaMemset(st->cerr, 0, sizeof(int)) != cudaSuccess) {
    free_nl(st);
    return nl_fail(SHF_ERR_CUDA, "nl_admm_init: cudaMemset");
  }
  cudaError_t e = cudaMemcpyAsync(st->f, f, sizeof(float) * P * C, cudaMemcpyDeviceToDevice, st->stream);
  if (e != cudaSuccess) {
    free_nl(st);
    return nl_fail(SHF_ERR_CUDA, std::string("nl_admm_init: ") + cudaGetErrorString(e));
  }
  rc = nl_restart(st);
  if (rc) {
    free_nl(st);
    return rc;
  }
  *out = st;
  return SHF_OK;
}

int nl_admm_reset(nl_state* st, const float* f, int f_on_host) {
  if (!st || !f) return nl_fail(SHF_ERR_ARG, "nl_admm_reset: NULL argument");
  if (!f_on_host && (reinterpret_cast<uintptr_t>(f) & 7u)) return nl_fail(SHF_ERR_ARG, "f must be 8-byte aligned");
  NL_CK(cudaMemcpyAsync(st->f, f, sizeof(float) * st->P() * st->C,
                        f_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st->stream));
  return nl_restart(st);
}

int nl_admm_graph(const nl_state* st, int* nbr, int* deg, int* solve_steps) {
  if (!st) return nl_fail(SHF_ERR_ARG, "nl_admm_graph: NULL state");
  if (nbr) std::copy(st->nbr_host.begin(), st->nbr_host.end(), nbr);
  if (deg) std::copy(st->deg_host.begin(), st->deg_host.end(), deg);
  if (solve_steps) *solve_steps = static_cast<int>(st->cheb_a.size());
  return SHF_OK;
}

int nl_admm_step(nl_state* st, int n) {
  if (!st || n < 0) return nl_fail(SHF_ERR_ARG, "nl_admm_step: bad argument");
  if (n == 0) return SHF_OK;
  if (!st->graph_tried) {
    st->graph_tried = true;
    cudaGraph_t graph = nullptr;
    if (st->stream && cudaStreamBeginCapture(st->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      cudaError_t e = enqueue_nl_iteration(st, nullptr);
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
      NL_CK(cudaGraphLaunch(st->exec, st->stream));
    else
      NL_CK(enqueue_nl_iteration(st, nullptr));
  }
  st->iter += n;
  return SHF_OK;
}

int nl_admm_kernel_times(nl_state* st, int n, float* ms, int* nk) {
  if (!st || !ms || n < 1) return nl_fail(SHF_ERR_ARG, "nl_admm_kernel_times: bad argument");
  cudaEvent_t ev[kNlKinds + 1];
  for (int i = 0; i <= kNlKinds; ++i) NL_CK(cudaEventCreate(&ev[i]));
  for (int i = 0; i < kNlKinds; ++i) ms[i] = 0.f;
  int rc = SHF_OK;
  for (int it = 0; it < n && rc == SHF_OK; ++it) {
    cudaError_t e = enqueue_nl_iteration(st, ev);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[kNlKinds]);
    for (int i = 0; i < kNlKinds && e == cudaSuccess; ++i) {
      float t = 0.f;
      e = cudaEventElapsedTime(&t, ev[i], ev[i + 1]);
      ms[i] += t / n;
    }
    if (e != cudaSuccess) rc = nl_fail(SHF_ERR_CUDA, std::string("nl_admm_kernel_times: ") + cudaGetErrorString(e));
  }
  for (int i = 0; i <= kNlKinds; ++i) cudaEventDestroy(ev[i]);
  if (rc == SHF_OK) st->iter += n;
  if (nk) *nk = kNlKinds;
  return rc;
}

const char* nl_admm_kernel_name(int i) { return (i >= 0 && i < kNlKinds) ? kNlNames[i] : ""; }

int nl_admm_get(nl_state* st, int what, void* dst, int on_host) {
  if (!st || !dst) return nl_fail(SHF_ERR_ARG, "nl_admm_get: NULL argument");
  const size_t P = st->P(), K = st->K, m = st->m;
  const cudaMemcpyKind kind = on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  switch (what) {
    case SEG_U: return nl_copy(st, dst, st->u, sizeof(float) * P * K, kind, on_host);
    case SEG_W: return nl_copy(st, dst, st->w, sizeof(float) * P * K, kind, on_host);
    case SEG_BW: return nl_copy(st, dst, st->bw, sizeof(float) * P * K, kind, on_host);
    case SEG_S: return nl_copy(st, dst, st->s, sizeof(float) * P * K, kind, on_host);
    case SEG_BV: return nl_copy(st, dst, st->bv, sizeof(float) * m * P * K, kind, on_host);
    case SEG_V: {  // v = d + b_v
      const size_t n = m * P * K;
      float* tgt = static_cast<float*>(dst);
      if (on_host) NL_CK(cudaMallocAsync(reinterpret_cast<void**>(&tgt), sizeof(float) * n, st->stream));
      k_nl_axpb<<<grid_for(n), kThreads, 0, st->stream>>>(st->d, st->bv, tgt, 1.f, n);
      cudaError_t e = cudaGetLastError();
      if (on_host) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(dst, tgt, sizeof(float) * n, cudaMemcpyDeviceToHost, st->stream);
        cudaError_t e2 = cudaFreeAsync(tgt, st->stream);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaStreamSynchronize(st->stream);
      }
      NL_CK(e);
      return SHF_OK;
    }
    case SEG_LABELS:
    case SEG_GAP: {
      NL_CK(shf::launch_labels(st->w, st->K, static_cast<int>(P), st->labels, st->gap, st->stream));
      return nl_copy(st, dst, what == SEG_LABELS ? static_cast<void*>(st->labels) : static_cast<void*>(st->gap),
                     sizeof(float) * P, kind, on_host);
    }
    case SEG_ENERGY: {
      k_nl_energy<<<kRedBlocks, kThreads, 0, st->stream>>>(st->w, st->s, st->nbr, st->deg, st->K, st->m, P,
                                                           st->red + 2);
      NL_CK(cudaGetLastError());
      k_nl_energy_final<<<1, 32, 0, st->stream>>>(st->red + 2, kRedBlocks, st->red);
      NL_CK(cudaGetLastError());
      double hst[2];
      NL_CK(cudaMemcpyAsync(hst, st->red, sizeof(hst), cudaMemcpyDeviceToHost, st->stream));
      NL_CK(cudaStreamSynchronize(st->stream));
      const double energy = hst[0] + static_cast<double>(st->lambda) * hst[1];
      if (on_host) {
        *static_cast<double*>(dst) = energy;
        return SHF_OK;
      }
      return nl_copy(st, dst, &energy, sizeof(double), cudaMemcpyHostToDevice, true);
    }
    case SEG_ITER: {
      if (!on_host) return nl_fail(SHF_ERR_ARG, "SEG_ITER is read into host memory");
      NL_CK(cudaStreamSynchronize(st->stream));
      *static_cast<int*>(dst) = st->iter;
      return SHF_OK;
    }
    default: return nl_fail(SHF_ERR_ARG, "nl_admm_get: unknown selector");
  }
}

int nl_admm_set(nl_state* st, int what, const void* src, int on_host) {
  if (!st || !src) return nl_fail(SHF_ERR_ARG, "nl_admm_set: NULL argument");
  const size_t P = st->P(), K = st->K, m = st->m;
  const cudaMemcpyKind kind = on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  int rc = SHF_OK;
  switch (what) {
    case SEG_W: rc = nl_copy(st, st->w, src, sizeof(float) * P * K, kind, false); break;
    case SEG_BW: rc = nl_copy(st, st->bw, src, sizeof(float) * P * K, kind, false); break;
    case SEG_U: rc = nl_copy(st, st->u, src, sizeof(float) * P * K, kind, false); break;
    case SEG_BV: rc = nl_copy(st, st->bv, src, sizeof(float) * m * P * K, kind, false); break;
    case SEG_V: {
      rc = nl_copy(st, st->d, src, sizeof(float) * m * P * K, kind, false);
      if (rc == SHF_OK) {
        k_nl_axpb<<<grid_for(m * P * K), kThreads, 0, st->stream>>>(st->d, st->bv, st->d, -1.f, m * P * K);
        NL_CK(cudaGetLastError());
      }
      break;
    }
    default: return nl_fail(SHF_ERR_ARG, "nl_admm_set: accepts SEG_W, SEG_BW, SEG_U, SEG_BV and SEG_V");
  }
  if (rc) return rc;
  NL_CK(rebuild_rhs(st));
  NL_CK(cudaStreamSynchronize(st->stream));
  return SHF_OK;
}

int nl_admm_sync(nl_state* st) {
  if (!st) return nl_fail(SHF_ERR_ARG, "nl_admm_sync: NULL state");
  NL_CK(cudaStreamSynchronize(st->stream));
  int gave_up = 0;
  NL_CK(cudaMemcpy(&gave_up, st->cerr, sizeof(int), cudaMemcpyDeviceToHost));
  if (gave_up) {
    NL_CK(cudaMemset(st->cerr, 0, sizeof(int)));
    return nl_fail(SHF_ERR_TIMEOUT, "nl_admm_sync: a grid barrier of the Chebyshev solve gave up");
  }
  return SHF_OK;
}

int nl_admm_barrier_selftest(nl_state* st) {
  if (!st) return nl_fail(SHF_ERR_ARG, "nl_admm_barrier_selftest: NULL state");
  NL_CK(cudaStreamSynchronize(st->stream));
  NL_CK(cudaMemsetAsync(st->cbar, 0, sizeof(unsigned), st->stream));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2);
  cfg.blockDim = dim3(32);
  cfg.stream = st->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  NL_CK(cudaLaunchKernelEx(&cfg, k_barrier_unreachable, st->cbar, st->cerr));
  return nl_admm_sync(st);
}

int nl_admm_destroy(nl_state* st) {
  free_nl(st);
  return SHF_OK;
}

}  // extern "C"

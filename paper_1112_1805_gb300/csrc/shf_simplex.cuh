// Pixelwise Euclidean projection onto the unit simplex (the w-step of the
// ADMM of Sec. 3), shared by the u/w-step kernels of both regularisers.
#pragma once

namespace shf {

// Projection of g[0..K) onto {x >= 0, sum x = 1}, as the paper constructs it:
// project onto the hyperplane sum = 1 (g + (1 - sum g)/q), set the negative
// components to zero and repeat on the remaining ones (at most K passes; the
// result is exact).  K <= KMAX <= 32.
template <int KMAX>
__device__ __forceinline__ void simplex_project(float (&g)[KMAX], int K) {
  unsigned act = (K >= 32) ? 0xffffffffu : ((1u << K) - 1u);
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

}  // namespace shf

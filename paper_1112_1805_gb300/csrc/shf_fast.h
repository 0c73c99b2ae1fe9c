// Fast path of the iteration (register FFTs, lengths R 2^a with R in {1, 3, 5}):
// interface between the host-side plan (shf_fast.cu) and the kernels, which
// live in shf_fast_col.cu (column transforms, per image height H) and
// shf_fast_row.cu (row transforms, per half width L), so that the two sets of
// template instances compile separately.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "shf_fft_reg.cuh"
#include "shf_internal.h"

// The supported transform lengths, for dispatch over template instances:
// rows (half widths L) up to 1024, columns (heights H) up to 2048.
#define SHF_FAST_SIZES(X) \
  X(8) X(16) X(24) X(32) X(40) X(48) X(64) X(80) X(96) X(128) X(160) X(192) X(256) X(320) X(384) X(512) X(640) X(768) X(1024)
#define SHF_COL_SIZES(X) SHF_FAST_SIZES(X) X(1280) X(1536) X(2048)

namespace shf {
namespace fast {

#ifdef __CUDACC__
// Programmatic dependent launch.  Every kernel of the iteration first builds
// what needs no earlier result (twiddle tables, constant operands), then waits
// for its predecessor grid to complete and flush (pdl_wait), and only then
// lets its own dependent launch (pdl_trigger).  So when a kernel starts, every
// grid before its immediate predecessor has completed, and the predecessor
// has passed its own wait.  Both are no-ops for a launch without the
// programmatic-serialization attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// L2 residency of a wave's coefficient spectra: the fan stores them with an
// evict-last policy (the v-step reads and rewrites them next), the gather,
// their last reader, loads them with an evict-first one (bezier512: gather
// 59.6 -> 56.3 us per launch, the iteration 2.3% shorter; the same policy on
// the v-step's stores slowed the v-step).
__device__ __forceinline__ uint64_t l2_evict_last_policy() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ void st_l2_hint(float2* p, float2 v, uint64_t policy) {
  asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(p), "f"(v.x), "f"(v.y), "l"(policy)
               : "memory");
}
__device__ __forceinline__ float2 ld_l2_hint(const float2* p, uint64_t policy) {
  float2 v;
  asm("ld.global.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(v.x), "=f"(v.y) : "l"(p), "l"(policy));
  return v;
}

__device__ __forceinline__ void load_table(float2* dst, const float2* __restrict__ src, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

// Launch with programmatic stream serialization: the kernel may start while
// its predecessor drains, and waits for it in pdl_wait.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

template <typename KERN>
cudaError_t allow_smem(KERN k, size_t bytes) {
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes));
}
#endif

// A wave of (label, filter) pairs: labels from l0, filters [f0, f0 + nf) of
// each; nv pairs in all, whose spectra are Y_v with v = (label - l0) nf + (f - f0).
struct Wave {
  int l0, f0, nf, nv;
};

// Column kernels (shf_fast_col.cu).  Whp: row pitch of the internal spectra.
// `variant` (ColKernel, shf_internal.h) selects the transform: 8 values per
// thread, or 16 (radix-16 passes; heights 512, 1024, 2048); 0 is the default
// for the height.
bool col_kernel_ok(int H, int variant);
cudaError_t prepare_col_kernels();
int col_ctas_per_sm(int H, int variant = 0);  // resident CTAs per SM of the gather kernel
int fan_ctas_per_sm(int H, int variant = 0);  // resident CTAs per SM of the fan kernel
// Ur [K][H][Wh] -> uhat [K][H][Whp]: column-forward of the row spectra of u.
cudaError_t col_fwd(const Geo& g, const float2* Ur, float2* uhat, int K, int Whp, cudaStream_t st);
// Y_v = column-inverse(W_f * uhat_label) on the (label, tile, filter) items of
// CTA ranges cta_begin[0..nc] of wave wv.
cudaError_t col_fan(const Geo& g, int nc, const float2* uhat, const WorkItem* items, const int* cta_begin,
                    float2* Y, int Whp, const Wave& wv, int variant, cudaStream_t st);
// partial[slot] = sum over runs of items of W_f * column-forward(Y_v).
cudaError_t col_gather(const Geo& g, int nc, const float2* Y, const WorkItem* items, const int* cta_begin,
                       float2* partial, int Whp, const Wave& wv, int variant, cudaStream_t st);
// T [K][H][Wh] = column-inverse of the per-(label, tile) sums of the partial slots.
cudaError_t col_reduce(const Geo& g, const float2* partial, const int* tile_begin, const int* tile_slots, float2* T,
                       int K, cudaStream_t st);

// Row kernels (shf_fast_row.cu).
cudaError_t prepare_row_kernels();
// Resident CTAs per SM and rows in flight per CTA of the v-step kernel
// (mode 0) or of its adjoint (mode 1).
// `variant` (RowKernel, shf_internal.h) selects the forward v-step: 8 values
// per thread, 16 (half widths 64..1024, powers of two) or pairs of rows (64,
// 128); 0 is the default for the width; the adjoint (mode 1) always takes its
// default.
bool row_kernel_ok(int L, int variant);
int row_ctas_per_sm(int L, int mode = 0, int variant = 0);
int row_groups_per_cta(int L, int mode = 0, int variant = 0);
// v-step on the rows of wave wv: ctas resident CTAs; code (optional,
// [K][eta][H][W] bytes) receives 0 where |g| < t, else sign g.
cudaError_t row_shrink(const Geo& g, int ctas, float2* Y, float* bv, const float* thr, int Whp, const Wave& wv,
                       float scale, signed char* code, int variant, cudaStream_t st);
// Adjoint of the v-step for the reverse mode: Y holds the spectra of the rows
// of S Qbar on input and those of the new bvbar on output; tpart
// [K][eta][H] receives the rows' threshold sums.
cudaError_t row_adjoint(const Geo& g, int ctas, float2* Y, float* bvbar, const float* thr, int Whp, const Wave& wv,
                        float scale, const signed char* code, double* tpart, cudaStream_t st);
// Shared memory of the u/w-step for K labels (0 if L is not supported).
size_t ustep_smem_bytes(int L, int K);
cudaError_t row_ustep(const Geo& g, const float2* T, const float* s, float* w, float* bw, float* u, float2* Ur, int K,
                      float gamma, float scale, cudaStream_t st);

}  // namespace fast
}  // namespace shf

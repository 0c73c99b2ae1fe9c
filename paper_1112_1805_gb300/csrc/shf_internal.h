// Internal interface between the C ABI layer and the kernel translation units.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "shf_fft.cuh"

struct shf_bank;

namespace shf {

constexpr int kMaxK = 16;     // labels per pixel held in registers by the w-step
constexpr int kMaxC = 3;      // image channels
constexpr int kMaxJ = 6;      // scales
constexpr int kMaxSide = 2048;
constexpr int kColThreads = 256;
constexpr int kRowThreads = 256;

// Geometry and launch shapes of one (H, W, J) problem.
struct Geo {
  int H, W, J, eta;
  int L;   // W / 2, length of the packed complex row transform
  int Wh;  // W / 2 + 1, columns of the half spectrum
  FftPlan planH, planL;
  int TC;       // columns per column-transform tile
  int ntiles;   // ceil(Wh / TC)
  int RB;       // rows per row-transform block
  int maxe;     // per-thread register elements of a column tile (8, 16 or 32)
  const float2* twH;  // exp(-2 pi i m / H), m < H
  const float2* twW;  // exp(-2 pi i m / W), m < W
  const float* bank;  // [eta][H][Wh]
  const int2* ranges; // [eta] first and last half-plane column where the filter is non-zero
};

// Filter descriptor in bank order: kind 0 low-pass, 1 horizontal cone,
// 2 vertical cone, 3 glued seam shearlet; scale j; shear k.
struct FilterDesc {
  int kind, j, k;
};

bool make_geo(int H, int W, int J, Geo* g);
int filter_descs(int J, FilterDesc* out);  // returns eta

// Filter bank and tables (shf_bank.cu).
cudaError_t launch_twiddles(float2* tw, int N, cudaStream_t st);
cudaError_t launch_build_bank(float* bank, const Geo& g, const FilterDesc* descs_dev, cudaStream_t st);
cudaError_t launch_filter_ranges(const float* bank, const Geo& g, int2* ranges, cudaStream_t st);
cudaError_t launch_data_term(const float* f, int C, const float* codebook_host, int K, float* s, int P,
                             cudaStream_t st);
cudaError_t launch_labels(const float* w, int K, int P, int* labels, float* gap, cudaStream_t st);
cudaError_t launch_count_nonfinite(const float* x, long n, int* count, cudaStream_t st);
// Deterministic sums: partial[block] in FP64 then one ordered final pass.
cudaError_t launch_dot(const float* a, const float* b, long n, double* partial, int nblocks, double* out,
                       cudaStream_t st);
cudaError_t launch_sqdiff(const float* a, const float* b, long n, double* partial, int nblocks, double* out,
                          cudaStream_t st);
cudaError_t launch_sum_partials(const double* partial, int n, double* out, cudaStream_t st);

// Transform kernels (shf_transform.cu).
// Real rows [planes][H][W] -> half spectra [planes][H][Wh] (row transforms).
cudaError_t run_row_r2c(const Geo& g, const float* in, float2* out, int planes, float scale, cudaStream_t st);
// Half spectra -> real rows, times `scale`.
cudaError_t run_row_c2r(const Geo& g, const float2* in, float* out, int planes, float scale, cudaStream_t st);
// ADMM v-step on coefficient spectra Y [nch*eta][H][Wh] (in place) and b_v.
// gout (optional): receives g = b_v + S u before the clipping, [planes][H][W].
cudaError_t run_row_shrink(const Geo& g, float2* Y, float* bv, const float* thr, int planes, float scale,
                           cudaStream_t st, float* gout = nullptr);
// sum_f lam[f] * ||ifft rows of Y_f||_1 into partial[nblocks] (nblocks returned).
cudaError_t run_row_l1(const Geo& g, const float2* Y, const float* lam, int planes, float scale, double* partial,
                       int* nblocks, cudaStream_t st);
// Column transform, fan-out over filters: in [nch][H][Wh] (row spectra) ->
// out [nch][eta][H][Wh] = column-inverse( W_f * column-forward(in) ).
cudaError_t run_col_fan(const Geo& g, const float2* in, float2* out, int nch, int groups, cudaStream_t st);
// Column transform, gather over filters: partial[grp][nch][H][Wh] =
// sum_{f in grp} W_f * column-forward(in[ch][f]).
cudaError_t run_col_gather(const Geo& g, const float2* in, float2* partial, int nch, int groups, cudaStream_t st);
// out[nch][H][Wh] = column-inverse( sum_grp partial[grp] ).
cudaError_t run_col_reduce_inv(const Geo& g, const float2* partial, float2* out, int nch, int groups,
                               cudaStream_t st);
// ADMM u-step and w-step per row block over all K labels.
cudaError_t run_row_ustep(const Geo& g, const float2* T, const float* s, float* w, float* bw, float* u, float2* Ur,
                          float* stv, int K, float gamma, float scale, cudaStream_t st);
int default_groups(const Geo& g, int nch);
// Sets the general path's tile shape (columns per column tile TC, rows per
// row block RB) in g when the kernels support it and their shared memory for
// K labels fits in `smem_limit` bytes; false (g unchanged) otherwise.
bool set_generic_tiles(Geo* g, int TC, int RB, int K, int smem_limit);
cudaError_t prepare_kernels();
int max_dynamic_smem_needed(const Geo& g, int K);
cudaError_t launch_sub(const float* a, const float* b, float* out, long n, cudaStream_t st);  // out = a - b

// Kinds of kernel launches in one ADMM iteration, for per-kernel timing.
enum KernelKind {
  kKindUstep = 0,
  kKindColFwd = 1,
  kKindFan = 2,
  kKindShrink = 3,
  kKindGather = 4,
  kKindReduce = 5,
  kKindEnd = 6,
  kNumKinds = 6
};

// Called before every launch of an iteration (and once with kKindEnd after the
// last), so that the caller can record an event there.
struct LaunchHook {
  void (*fn)(void* ctx, int kind) = nullptr;
  void* ctx = nullptr;
  void mark(int kind) const {
    if (fn) fn(ctx, kind);
  }
};

// Static work list of the fast path.  A wave is a set of (label, filter)
// pairs whose coefficient spectra stay in L2 between its three launches: the
// filters [f0, f0 + nf) of one label when a label's spectra exceed the wave
// budget, else whole labels [l0, l0 + nl) (nf = eta), so that small images
// fill the GPU with fewer, larger launches.  The wave's spectra are indexed by
// v = (label - l0) nf + (f - f0).  Its (label, column tile, filter) items whose
// filter support touches the tile (fast_tile(g) half-spectrum columns) are
// listed in that order and cut into one contiguous, balanced range per CTA of
// a column launch (separately for the fan and the gather, which run different
// numbers of resident CTAs).  Within a CTA's
// range, each run of one (label, tile) is one partial-sum slot of the
// synthesis; the slots of a (label, tile) are summed in filter order.
struct WorkItem {
  int tile;    // column tile
  int filter;  // filter index (0..eta-1)
  int slot;    // partial-sum slot of the item's run
  int label;
};
constexpr int kDefaultWaveMiB = 128;  // coefficient spectra per wave
// FFT kernel variants of a plan (0: the default for the size).
enum RowKernel { kRowDefault = 0, kRow8 = 1, kRow16 = 2, kRowPair = 3, kRowV = 4 };
enum ColKernel { kColDefault = 0, kCol8 = 1, kCol16 = 2, kColV = 3 };
struct FastPlan {
  int wave_mib = kDefaultWaveMiB;
  int col_ctas_per_sm = 0;  // CTAs per SM of the column launches (0: as many as fit)
  int row_kernel = kRowDefault;  // forward v-step transform (RowKernel)
  int col_kernel = kColDefault;  // fan and gather transforms (ColKernel)
  int serial = 0;           // 1: launches without programmatic dependent launch
  int sms = 0;              // SMs the fan, v-step and gather grids are sized for (0: all)
  int col_ctas = 0;         // resolved: CTAs of one gather launch
  int fan_ctas = 0;         // resolved: CTAs of one fan launch (all resident)
  int row_ctas = 0;         // resolved: resident CTAs of the row (v-step) launch
  std::vector<int> wave_l0, wave_nl;  // per wave: first label, number of labels
  std::vector<int> wave_f0, wave_nf;  // per wave: first filter, number of filters
  std::vector<int> wave_cta0;         // per wave: first entry of its gather ranges in cta_begin (size waves + 1)
  std::vector<int> wave_fcta0;        // per wave: first entry of its fan ranges in cta_begin (size waves + 1)
  int y_planes = 0;                   // spectra planes of the largest wave (max nl nf)
  int nslots = 0;                     // partial slots in all (every wave and label)
  const WorkItem* items = nullptr;    // device, all waves
  const int* cta_begin = nullptr;     // device, item range [cta_begin[c], cta_begin[c+1]) of CTA c
  const int* tile_begin = nullptr;    // device [K ntiles + 1], into tile_slots, per (label, tile)
  const int* tile_slots = nullptr;    // device, slots of each (label, tile) in filter order
};

// Whether launch_pdl asks for programmatic dependent launch, per host thread
// (on unless a PdlScope turned it off).  It lets a kernel's CTAs become
// resident and run their prologue while the previous kernel drains; at some
// shapes that costs more than it saves (a plan's `serial` field).  Kernels
// launched through fast::launch_pdl read it.
inline bool& pdl_enabled() {
  static thread_local bool on = true;
  return on;
}
struct PdlScope {
  bool old;
  explicit PdlScope(bool on) : old(pdl_enabled()) { pdl_enabled() = on; }
  ~PdlScope() { pdl_enabled() = old; }
  PdlScope(const PdlScope&) = delete;
  PdlScope& operator=(const PdlScope&) = delete;
};

// Fast path for power-of-two sizes (shf_fast.cu).
bool fast_path_ok(const Geo& g);
int fast_tile(const Geo& g);  // columns per tile of the fast column kernels (8, or 4 for H > 1024)
cudaError_t prepare_fast_kernels();
int fast_wave(const Geo& g, int wave_mib);  // filters per wave of one label (at most eta)
int fast_wave_labels(const Geo& g, int wave_mib, int K);  // labels per wave (1: waves of filters)
int fast_pitch(const Geo& g);       // row pitch (complex) of the internal spectra: Wh rounded up to 8
bool fast_ustep_ok(const Geo& g, int K);
// u-step, w-step, b_w update and row spectra of u (power-of-two sizes, K <= 8).
cudaError_t run_fast_ustep(const Geo& g, const float2* T, const float* s, float* w, float* bw, float* u, float2* Ur,
                           int K, float gamma, float scale, cudaStream_t st);
// Everything of an iteration after the u/w-step: Ur (row spectra of u) -> uhat
// -> per-filter analysis, v-step and synthesis -> T.
// code (optional, [K][eta][H][W] bytes): receives, per coefficient, 0 where
// |g| < t_f and the sign of g elsewhere (for the reverse mode).
cudaError_t run_fast_iteration_body(const Geo& g, const FastPlan& plan, const float2* Ur, float2* uhat, float2* Y,
                                    float* bv, const float* thr, float2* partial, float2* T, int K, float scale,
                                    cudaStream_t st, const LaunchHook& hook, signed char* code = nullptr);
// Adjoint of the analysis - v-step - synthesis part of an iteration (reverse
// mode): Qr [K][H][Wh] the row spectra of Qbar; bvbar [K][eta][H][W] updated in
// place with the codes of the forward iteration; Tbar [K][H][Wh] receives the
// column-inverse spectrum of S^T bvbar (row-inverse and 1/(HW) left to the
// caller); tpart [K][eta][H] the rows' threshold sums.
cudaError_t run_fast_adjoint_body(const Geo& g, const FastPlan& plan, const float2* Qr, float2* uhat, float2* Y,
                                  float* bvbar, const float* thr, float2* partial, float2* Tbar, int K, float scale,
                                  const signed char* code, double* tpart, cudaStream_t st);
// Resident CTAs of one gather launch for `per_sm` CTAs per SM (0: as many
// as fit; larger values are clamped to that), and of one fan launch, on `sms`
// SMs (0, or more than the device has: all of them).
int fast_col_ctas(const Geo& g, int per_sm, int col_kernel = kColDefault, int sms = 0);
int fast_fan_ctas(const Geo& g, int col_kernel = kColDefault, int sms = 0);
bool fast_row_kernel_ok(const Geo& g, int row_kernel);
bool fast_col_kernel_ok(const Geo& g, int col_kernel);
// Resident CTAs of the row (v-step) kernel on `sms` SMs (0: all).
int fast_row_ctas(const Geo& g, int row_kernel = kRowDefault, int sms = 0);
// Host construction of the work list of K labels from the filters' column
// ranges (ranges_host[eta]) for plan->wave_mib and plan->col_ctas; returns the
// host arrays to upload (cta_begin holds one entry more per wave).
void build_fast_plan(const Geo& g, const int2* ranges_host, int K, FastPlan* plan, std::vector<WorkItem>* items,
                     std::vector<int>* cta_begin, std::vector<int>* tile_begin, std::vector<int>* tile_slots);

// Reverse mode of the unrolled iteration (shf_adjoint.cu).
// gwbar = bwbar + J_P(wbar - bwbar), J_P the projection onto the face of the
// simplex where w' > 0.
cudaError_t launch_adj_proj(const float* wn, const float* wbar, const float* bwbar, float* gwbar, int K, int P,
                            cudaStream_t st);
// bvbar <- dbar (1 - 2m) + bvbar m with m = [|g| < t_f]; per-filter sums of
// sign(g)(1 - m)(bvbar - 2 dbar) accumulated (fixed order, FP64) into tbar[eta].
cudaError_t launch_adj_shrink(const float* g, const float* dbar, float* bvbar, const float* thr, int K, int eta,
                              long P, double* tpart, double* tbar, cudaStream_t st);
// ub = gwbar + st; Qbar = ub/2; wbar = ub/2; bwbar = gwbar - ub/2; sbar += -gamma ub/2.
cudaError_t launch_adj_u(const float* gwbar, const float* st_, float* Qbar, float* wbar, float* bwbar, float* sbar,
                         float gamma, long n, cudaStream_t st);
// dL/dc[k][ch] = sum_x sbar_k (-2)(f_ch - c_k,ch) (FP64, fixed order) into
// out_host; dL/df (optional, device) = sum_k sbar_k 2 (f_ch - c_k,ch).
cudaError_t adj_codebook(const float* sbar, const float* f, const float* codebook_host, int K, int C, long P,
                         double* part, double* out_dev, float* fbar, cudaStream_t st);
int adj_part_blocks();
// tbar[f] += sum over labels and rows of tpart[(k eta + f) H + row], in order.
cudaError_t launch_adj_tsum_rows(const double* tpart, int K, int eta, int H, double* tbar, cudaStream_t st);

// The TV u-step on register FFTs (shf_tv_fast.cu) for W/2 in 64..1024 and H
// in 512, 1024, 2048 (powers of two): spectra [K][H][tv_fast_pitch(W)].
namespace tvfast {
bool tv_fast_ok(int H, int W);
int tv_fast_pitch(int W);
cudaError_t tv_fast_prepare();
// rhs = q + grad^T d row by row, row transforms -> half spectra Ur.
cudaError_t tv_fast_rows_fwd(const float* q, const float* d, float2* Ur, int K, int H, int W, const float2* twW,
                             cudaStream_t st);
// column transform, times the inverse symbol sym [H][W/2+1], inverse column transform: Ur -> Y.
cudaError_t tv_fast_cols(const float2* Ur, const float* sym, float2* Y, int K, int H, int W, const float2* twH,
                         cudaStream_t st);
// inverse row transforms times scale -> u [K][H][W].
cudaError_t tv_fast_rows_inv(const float2* Y, float* u, int K, int H, int W, float scale, const float2* twW,
                             cudaStream_t st);
}  // namespace tvfast

// C ABI layer (shf_capi.cu): the geometry and device tables of a bank, and the
// thread-local message behind shf_last_error() (returns code).
void bank_geo(const shf_bank* b, Geo* g);
int bank_device(const shf_bank* b);  // the device the bank's tables live on
int set_error(int code, const std::string& msg);

}  // namespace shf

// C ABI of the shearlet segmentation library: filter banks, the shearlet
// transform and the ADMM state (Haeuser & Steidl, arXiv:1112.1805).  Argument
// checking, buffer ownership, CUDA-graph capture of one ADMM iteration,
// readouts and checkpoints.  All arithmetic runs in the kernels of
// shf_bank.cu and shf_transform.cu.
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "shearseg.h"
#include "shf_internal.h"

using shf::Geo;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

#define SHF_CK(call)                                                                              \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess) return fail(SHF_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

bool aligned8(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 7u) == 0; }

template <typename T>
int dev_alloc(T** p, size_t count, const char* what) {
  *p = nullptr;
  if (count == 0) return SHF_OK;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(e == cudaErrorMemoryAllocation ? SHF_ERR_OOM : SHF_ERR_CUDA,
                std::string("cudaMalloc(") + what + "): " + cudaGetErrorString(e));
  }
  return SHF_OK;
}

int check_sizes(int H, int W, int J) {
  if (J < 1 || J > shf::kMaxJ) return fail(SHF_ERR_ARG, "J must be in [1, 6]");
  if (H < 8 || W < 8 || H > shf::kMaxSide || W > shf::kMaxSide)
    return fail(SHF_ERR_SIZE, "H and W must be in [8, 2048]");
  if (W & 1) return fail(SHF_ERR_SIZE, "W must be even");
  shf::FftPlan p;
  if (!shf::make_plan(H, &p) || !shf::make_plan(W / 2, &p))
    return fail(SHF_ERR_SIZE, "H and W/2 must be products of powers of 2, 3 and 5");
  return SHF_OK;
}

}  // namespace

struct shf_bank {
  Geo g;
  float* bank = nullptr;
  int2* ranges = nullptr;
  float2* twH = nullptr;
  float2* twW = nullptr;
  shf::FilterDesc* descs = nullptr;
  int device = 0;
};

struct seg_state {
  const shf_bank* bank = nullptr;
  seg_batch* batch = nullptr;  // the batch whose graphs replay this state, if any
  Geo g;
  int K = 0, C = 0;
  float gamma = 1.f;
  std::vector<float> Lambda;
  std::vector<float> codebook;  // [K][C], host copy for seg_admm_reset
  int max_iters = 0;
  float tol = 0.f;
  int check_every = 1;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  float *f = nullptr, *s = nullptr, *bv = nullptr, *w = nullptr, *bw = nullptr, *u = nullptr, *stv = nullptr;
  float2 *Ur = nullptr, *Y = nullptr, *partial = nullptr, *T = nullptr;
  float *thr = nullptr, *lam = nullptr, *gap = nullptr;
  int* labels = nullptr;
  int* flag = nullptr;
  double* red = nullptr;
  int red_len = 0;
  int groups = 1;
  cudaGraphExec_t exec = nullptr;        // one iteration
  cudaGraphExec_t exec_timed = nullptr;  // the same with an event before every launch
  bool graph_tried = false;
  bool untimed = false;  // steps record no per-kernel events (the tuner's trials)
  bool fast = false;          // power-of-two sizes: the shf_fast.cu kernels
  bool fast_ustep = false;    // ... including the u/w-step (K <= 8)
  shf::FastPlan plan;         // fast path: static per-wave work list
  std::vector<int2> ranges_host;  // fast path: the filters' column ranges
  shf::WorkItem* d_items = nullptr;
  int *d_cta_begin = nullptr, *d_tile_begin = nullptr, *d_tile_slots = nullptr;
  float2* uhat = nullptr;     // fast path: 2-D spectra of u [K][H][Wh]
  // Events recorded before every launch of an iteration (graph event nodes),
  // with the kind of the launch that follows each.
  // created when a timed iteration is first captured, as many as it has marks
  static constexpr int kMaxMarks = 8192;
  std::vector<cudaEvent_t> ev;
  std::vector<int> kinds;
  int nmarks = 0;
  bool marks_ok = true;
  // unrolled mode (reverse-mode differentiation): generic-path scratch and
  // the states kept every un_ck iterations
  int un_T = 0, un_ck = 0;
  float2* un_Y = nullptr;        // [K][eta][H][Wh]
  float2* un_partial = nullptr;  // [un_groups][K][H][Wh]
  int un_groups = 0;
  std::vector<float*> ck_bv, ck_w, ck_bw;
  std::vector<float2*> ck_T;
  // the forward and reverse sweeps captured as graphs for (T, ckpt) = un_key;
  // the reverse sweep's temporaries live in un_mem (un_mem_bytes)
  cudaGraphExec_t un_fwd_exec = nullptr, un_bwd_exec = nullptr;
  int un_fwd_key[2] = {0, 0}, un_bwd_key[2] = {0, 0};
  char* un_mem = nullptr;
  size_t un_mem_bytes = 0;
  bool un_bwd_pending = false;  // a reverse sweep was enqueued (its results are in un_mem)
  long long iter = 0;
  size_t P() const { return static_cast<size_t>(g.H) * g.W; }
  size_t Ph() const { return static_cast<size_t>(g.H) * g.Wh; }
};

namespace shf {
void bank_geo(const shf_bank* b, Geo* g) { *g = b->g; }
int bank_device(const shf_bank* b) { return b->device; }
int set_error(int code, const std::string& msg) { return fail(code, msg); }
}  // namespace shf

extern "C" {

int shf_version(void) { return 100; }

const char* shf_last_error(void) { return g_err.c_str(); }

int shfilters_build(int H, int W, int J, void* stream, shf_bank** out) {
  if (!out) return fail(SHF_ERR_ARG, "out is NULL");
  *out = nullptr;
  int rc = check_sizes(H, W, J);
  if (rc) return rc;
  Geo g;
  if (!shf::make_geo(H, W, J, &g)) return fail(SHF_ERR_SIZE, "unsupported geometry");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int device = 0, optin = 0;
  SHF_CK(cudaGetDevice(&device));
  SHF_CK(shf::prepare_kernels());
  SHF_CK(shf::prepare_fast_kernels());
  SHF_CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
  if (shf::max_dynamic_smem_needed(g, shf::kMaxK) > optin)
    return fail(SHF_ERR_SIZE, "tile does not fit in shared memory");
  auto* b = new shf_bank();
  b->g = g;
  b->device = device;
  std::vector<shf::FilterDesc> d(g.eta);
  shf::filter_descs(J, d.data());
  if ((rc = dev_alloc(&b->bank, static_cast<size_t>(g.eta) * H * g.Wh, "bank")) ||
      (rc = dev_alloc(&b->twH, H, "twH")) || (rc = dev_alloc(&b->twW, W, "twW")) ||
      (rc = dev_alloc(&b->descs, g.eta, "descs")) || (rc = dev_alloc(&b->ranges, g.eta, "ranges"))) {
    shfilters_destroy(b);
    return rc;
  }
  b->g.bank = b->bank;
  b->g.ranges = b->ranges;
  b->g.twH = b->twH;
  b->g.twW = b->twW;
  cudaError_t e = cudaMemcpyAsync(b->descs, d.data(), sizeof(shf::FilterDesc) * g.eta, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = shf::launch_twiddles(b->twH, H, st);
  if (e == cudaSuccess) e = shf::launch_twiddles(b->twW, W, st);
  if (e == cudaSuccess) e = shf::launch_build_bank(b->bank, b->g, b->descs, st);
  if (e == cudaSuccess) e = shf::launch_filter_ranges(b->bank, b->g, b->ranges, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // d is a host temporary
  if (e != cudaSuccess) {
    shfilters_destroy(b);
    return fail(SHF_ERR_CUDA, std::string("shfilters_build: ") + cudaGetErrorString(e));
  }
  *out = b;
  return SHF_OK;
}

int shfilters_destroy(shf_bank* b) {
  if (!b) return SHF_OK;
  cudaDeviceSynchronize();
  cudaFree(b->bank);
  cudaFree(b->twH);
  cudaFree(b->twW);
  cudaFree(b->descs);
  cudaFree(b->ranges);
  delete b;
  return SHF_OK;
}

int shfilters_info(const shf_bank* b, int* eta, int* H, int* W, int* J) {
  if (!b) return fail(SHF_ERR_ARG, "bank is NULL");
  if (eta) *eta = b->g.eta;
  if (H) *H = b->g.H;
  if (W) *W = b->g.W;
  if (J) *J = b->g.J;
  return SHF_OK;
}

int shfilters_copy(const shf_bank* b, float* dst, void* stream) {
  if (!b || !dst) return fail(SHF_ERR_ARG, "NULL argument");
  SHF_CK(cudaMemcpyAsync(dst, b->bank, sizeof(float) * b->g.eta * b->g.H * b->g.Wh, cudaMemcpyDeviceToDevice,
                         static_cast<cudaStream_t>(stream)));
  return SHF_OK;
}

int shearlet_analyze(const shf_bank* b, const float* u, int nch, float* coef, void* stream) {
  if (!b || !u || !coef || nch < 1) return fail(SHF_ERR_ARG, "shearlet_analyze: bad argument");
  if (!aligned8(u) || !aligned8(coef)) return fail(SHF_ERR_ARG, "shearlet_analyze: pointers must be 8-byte aligned");
  const Geo& g = b->g;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t ph = static_cast<size_t>(g.H) * g.Wh;
  float2* tmp = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&tmp), sizeof(float2) * ph * nch * (1 + g.eta), st);
  if (e != cudaSuccess) return fail(SHF_ERR_OOM, std::string("shearlet_analyze: ") + cudaGetErrorString(e));
  float2* Ur = tmp;
  float2* Y = tmp + ph * nch;
  e = shf::run_row_r2c(g, u, Ur, nch, 1.f, st);
  if (e == cudaSuccess) e = shf::run_col_fan(g, Ur, Y, nch, shf::default_groups(g, nch), st);
  if (e == cudaSuccess) e = shf::run_row_c2r(g, Y, coef, nch * g.eta, 1.f / (static_cast<float>(g.H) * g.W), st);
  cudaError_t e2 = cudaFreeAsync(tmp, st);
  if (e != cudaSuccess || e2 != cudaSuccess)
    return fail(SHF_ERR_CUDA, std::string("shearlet_analyze: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
  return SHF_OK;
}

namespace {
// T[nch][H][Wh] = column-inverse of sum_f W_f * fft2(coef_f) (unscaled).
cudaError_t synthesis_spectrum(const Geo& g, const float* coef, int nch, float2* T, cudaStream_t st) {
  const size_t ph = static_cast<size_t>(g.H) * g.Wh;
  const int groups = shf::default_groups(g, nch);
  float2* tmp = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&tmp), sizeof(float2) * ph * nch * (g.eta + groups), st);
  if (e != cudaSuccess) return e;
  float2* Z = tmp;
  float2* part = tmp + ph * nch * g.eta;
  e = shf::run_row_r2c(g, coef, Z, nch * g.eta, 1.f, st);
  if (e == cudaSuccess) e = shf::run_col_gather(g, Z, part, nch, groups, st);
  if (e == cudaSuccess) e = shf::run_col_reduce_inv(g, part, T, nch, groups, st);
  cudaError_t e2 = cudaFreeAsync(tmp, st);
  return e != cudaSuccess ? e : e2;
}
}  // namespace

int shearlet_synthesize(const shf_bank* b, const float* coef, int nch, float* u, void* stream) {
  if (!b || !coef || !u || nch < 1) return fail(SHF_ERR_ARG, "shearlet_synthesize: bad argument");
  if (!aligned8(u) || !aligned8(coef))
    return fail(SHF_ERR_ARG, "shearlet_synthesize: pointers must be 8-byte aligned");
  const Geo& g = b->g;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t ph = static_cast<size_t>(g.H) * g.Wh;
  float2* T = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&T), sizeof(float2) * ph * nch, st);
  if (e != cudaSuccess) return fail(SHF_ERR_OOM, std::string("shearlet_synthesize: ") + cudaGetErrorString(e));
  e = synthesis_spectrum(g, coef, nch, T, st);
  if (e == cudaSuccess) e = shf::run_row_c2r(g, T, u, nch, 1.f / (static_cast<float>(g.H) * g.W), st);
  cudaError_t e2 = cudaFreeAsync(T, st);
  if (e != cudaSuccess || e2 != cudaSuccess)
    return fail(SHF_ERR_CUDA, std::string("shearlet_synthesize: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
  return SHF_OK;
}

// ---------------------------------------------------------------------------
// ADMM state
// ---------------------------------------------------------------------------

namespace {

void free_state(seg_state* s) {
  if (s->exec) cudaGraphExecDestroy(s->exec);
  if (s->exec_timed) cudaGraphExecDestroy(s->exec_timed);
  for (cudaEvent_t e : s->ev)
    if (e) cudaEventDestroy(e);
  cudaFree(s->uhat);
  cudaFree(s->d_items);
  cudaFree(s->d_cta_begin);
  cudaFree(s->d_tile_begin);
  cudaFree(s->d_tile_slots);
  cudaFree(s->un_Y);
  cudaFree(s->un_partial);
  if (s->un_fwd_exec) cudaGraphExecDestroy(s->un_fwd_exec);
  if (s->un_bwd_exec) cudaGraphExecDestroy(s->un_bwd_exec);
  cudaFree(s->un_mem);
  for (float* p : s->ck_bv) cudaFree(p);
  for (float* p : s->ck_w) cudaFree(p);
  for (float* p : s->ck_bw) cudaFree(p);
  for (float2* p : s->ck_T) cudaFree(p);
  float* fl[] = {s->f, s->s, s->bv, s->w, s->bw, s->u, s->stv, s->thr, s->lam, s->gap};
  for (float* p : fl) cudaFree(p);
  cudaFree(s->Ur);
  cudaFree(s->Y);
  cudaFree(s->partial);
  cudaFree(s->T);
  cudaFree(s->labels);
  cudaFree(s->flag);
  cudaFree(s->red);
  if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
  delete s;
}

// Data term from st->f and a zero state; checks f for NaN/Inf (synchronises).
int restart(seg_state* st, const float* codebook) {
  const Geo& g = st->g;
  const size_t P = st->P();
  SHF_CK(cudaMemsetAsync(st->flag, 0, sizeof(int), st->stream));
  SHF_CK(shf::launch_count_nonfinite(st->f, static_cast<long>(P * st->C), st->flag, st->stream));
  if (codebook) SHF_CK(shf::launch_data_term(st->f, st->C, codebook, st->K, st->s, static_cast<int>(P), st->stream));
  SHF_CK(cudaMemsetAsync(st->bv, 0, sizeof(float) * P * st->K * g.eta, st->stream));
  SHF_CK(cudaMemsetAsync(st->w, 0, sizeof(float) * P * st->K, st->stream));
  SHF_CK(cudaMemsetAsync(st->bw, 0, sizeof(float) * P * st->K, st->stream));
  SHF_CK(cudaMemsetAsync(st->u, 0, sizeof(float) * P * st->K, st->stream));
  SHF_CK(cudaMemsetAsync(st->T, 0, sizeof(float2) * st->Ph() * st->K, st->stream));
  int bad = 0;
  SHF_CK(cudaMemcpyAsync(&bad, st->flag, sizeof(int), cudaMemcpyDeviceToHost, st->stream));
  SHF_CK(cudaStreamSynchronize(st->stream));
  st->iter = 0;
  if (bad) return fail(SHF_ERR_NONFINITE, "image contains NaN or Inf");
  return SHF_OK;
}

// Launches of one iteration, plus the closing mark.
int marks_needed(const seg_state* st) {
  if (!st->fast) return 8;
  int n = 4;  // u/w-step, column forward, reduction, end
  n += 3 * static_cast<int>(st->plan.wave_f0.size());  // fan, v-step, gather per wave
  return n;
}

// Creates the timing events an iteration of the current plan needs (at most
// kMaxMarks); a failure leaves the timing disabled.
void ensure_marks(seg_state* st) {
  const size_t need = static_cast<size_t>(std::min(marks_needed(st), static_cast<int>(seg_state::kMaxMarks)));
  while (st->ev.size() < need) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      break;
    }
    st->ev.push_back(e);
  }
  st->kinds.resize(st->ev.size());
}

// Records the event of the next mark; during stream capture it becomes an
// event-record node of the graph (cudaEventRecordExternal), so that each
// replay timestamps it.  A failed record only disables the timing (its error
// is cleared, not left for a later call to report).
void mark_launch(void* ctx, int kind) {
  auto* st = static_cast<seg_state*>(ctx);
  if (st->nmarks >= static_cast<int>(st->ev.size())) {
    st->marks_ok = false;
    return;
  }
  const int i = st->nmarks++;
  st->kinds[i] = kind;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(st->stream, &cs);
  if (e == cudaSuccess)
    e = cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(st->ev[i], st->stream, cudaEventRecordExternal)
                                            : cudaEventRecord(st->ev[i], st->stream);
  if (e != cudaSuccess) {
    st->marks_ok = false;
    cudaGetLastError();
  }
}

// One ADMM iteration; `timed`: with an event recorded before every launch and
// after the last one; `code` (fast path, optional): the per-coefficient codes
// of the v-step for the reverse mode.
cudaError_t enqueue_iteration(seg_state* st, bool timed, signed char* code = nullptr) {
  const Geo& g = st->g;
  const shf::PdlScope pdl(!(st->fast && st->plan.serial));
  const float scale = 1.f / (static_cast<float>(g.H) * g.W);
  cudaStream_t s = st->stream;
  shf::LaunchHook hook;
  if (timed) {
    hook.fn = mark_launch;
    hook.ctx = st;
    st->nmarks = 0;
    st->marks_ok = true;
  }
  hook.mark(shf::kKindUstep);
  cudaError_t e =
      st->fast_ustep
          ? shf::run_fast_ustep(g, st->T, st->s, st->w, st->bw, st->u, st->Ur, st->K, st->gamma, scale, s)
          : shf::run_row_ustep(g, st->T, st->s, st->w, st->bw, st->u, st->Ur, nullptr, st->K, st->gamma, scale, s);
  if (st->fast) {
    if (e == cudaSuccess)
      e = shf::run_fast_iteration_body(g, st->plan, st->Ur, st->uhat, st->Y, st->bv, st->thr, st->partial, st->T,
                                       st->K, scale, s, hook, code);
  } else {
    hook.mark(shf::kKindFan);
    if (e == cudaSuccess) e = shf::run_col_fan(g, st->Ur, st->Y, st->K, st->groups, s);
    hook.mark(shf::kKindShrink);
    if (e == cudaSuccess) e = shf::run_row_shrink(g, st->Y, st->bv, st->thr, st->K * g.eta, scale, s);
    hook.mark(shf::kKindGather);
    if (e == cudaSuccess) e = shf::run_col_gather(g, st->Y, st->partial, st->K, st->groups, s);
    hook.mark(shf::kKindReduce);
    if (e == cudaSuccess) e = shf::run_col_reduce_inv(g, st->partial, st->T, st->K, st->groups, s);
  }
  hook.mark(shf::kKindEnd);
  return e;
}

// One iteration on the generic kernels with the full coefficient scratch of
// the unrolled mode; gout (optional) records g = b_v + S u.
cudaError_t enqueue_generic_iteration(seg_state* st, float* gout) {
  const Geo& g = st->g;
  const float scale = 1.f / (static_cast<float>(g.H) * g.W);
  cudaStream_t s = st->stream;
  cudaError_t e =
      shf::run_row_ustep(g, st->T, st->s, st->w, st->bw, st->u, st->Ur, nullptr, st->K, st->gamma, scale, s);
  if (e == cudaSuccess) e = shf::run_col_fan(g, st->Ur, st->un_Y, st->K, st->groups, s);
  if (e == cudaSuccess) e = shf::run_row_shrink(g, st->un_Y, st->bv, st->thr, st->K * g.eta, scale, s, gout);
  if (e == cudaSuccess) e = shf::run_col_gather(g, st->un_Y, st->un_partial, st->K, st->un_groups, s);
  if (e == cudaSuccess) e = shf::run_col_reduce_inv(g, st->un_partial, st->T, st->K, st->un_groups, s);
  return e;
}

cudaGraphExec_t capture_iteration(seg_state* st, bool timed) {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  if (cudaStreamBeginCapture(st->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  cudaError_t e = enqueue_iteration(st, timed);
  cudaError_t e2 = cudaStreamEndCapture(st->stream, &graph);
  if (e == cudaSuccess && e2 == cudaSuccess && graph && (!timed || st->marks_ok)) {
    if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) exec = nullptr;
  }
  if (graph) cudaGraphDestroy(graph);
  cudaGetLastError();
  return exec;
}

// Captures one iteration into two graphs (plain, and with the timing events)
// when the stream can be captured (not the legacy default stream); otherwise
// iterations are launched directly.  An iteration with more launches than
// timing marks keeps only the plain graph (seg_admm_kernel_times then reports
// the timing as unavailable).
void try_capture(seg_state* st) {
  st->graph_tried = true;
  ensure_marks(st);
  if (st->stream == nullptr) return;
  st->exec = capture_iteration(st, false);
  if (st->exec) st->exec_timed = capture_iteration(st, true);
}

void drop_batch_graphs(seg_batch* b);

void drop_graphs(seg_state* st) {
  // a batch's graphs hold this state's buffers: they go too (a new plan
  // reallocates them)
  if (st->batch) drop_batch_graphs(st->batch);
  if (st->exec) cudaGraphExecDestroy(st->exec);
  if (st->exec_timed) cudaGraphExecDestroy(st->exec_timed);
  if (st->un_fwd_exec) cudaGraphExecDestroy(st->un_fwd_exec);
  if (st->un_bwd_exec) cudaGraphExecDestroy(st->un_bwd_exec);
  st->exec = st->exec_timed = st->un_fwd_exec = st->un_bwd_exec = nullptr;
  st->un_fwd_key[0] = st->un_fwd_key[1] = st->un_bwd_key[0] = st->un_bwd_key[1] = 0;
  st->graph_tried = false;
}

// Captures the work `enqueue` puts on the state's stream into an executable
// graph; nullptr when the stream cannot be captured or the work failed.
extern "C++" template <typename F>
cudaGraphExec_t capture_work(seg_state* st, F enqueue) {
  if (st->stream == nullptr) return nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  if (cudaStreamBeginCapture(st->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  cudaError_t e = enqueue();
  cudaError_t e2 = cudaStreamEndCapture(st->stream, &graph);
  if (e == cudaSuccess && e2 == cudaSuccess && graph && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess)
    exec = nullptr;
  if (graph) cudaGraphDestroy(graph);
  cudaGetLastError();
  return exec;
}

// Fast path: builds the work list for (wave_mib, col_ctas_per_sm) and
// allocates what depends on it (one wave of coefficient spectra Y, the
// partial tiles, the device work list); the previous buffers are released
// only once the new ones exist.  Synchronises the state's stream.
int install_fast_plan(seg_state* st, int wave_mib, int col_ctas_per_sm, int row_kernel = shf::kRowDefault,
                      int col_kernel = shf::kColDefault, int serial = 0, int sms = 0) {
  const Geo& g = st->g;
  shf::FastPlan plan;
  plan.wave_mib = wave_mib;
  plan.col_ctas_per_sm = col_ctas_per_sm;
  plan.row_kernel = row_kernel;
  plan.col_kernel = col_kernel;
  plan.serial = serial;
  plan.sms = sms;
  plan.col_ctas = shf::fast_col_ctas(g, col_ctas_per_sm, col_kernel, sms);
  plan.fan_ctas = shf::fast_fan_ctas(g, col_kernel, sms);
  plan.row_ctas = shf::fast_row_ctas(g, row_kernel, sms);
  if (plan.col_ctas < 1 || plan.fan_ctas < 1 || plan.row_ctas < 1)
    return fail(SHF_ERR_CUDA, "install_fast_plan: no resident CTA");
  std::vector<shf::WorkItem> h_items;
  std::vector<int> h_cta_begin, h_tile_begin, h_tile_slots;
  shf::build_fast_plan(g, st->ranges_host.data(), st->K, &plan, &h_items, &h_cta_begin, &h_tile_begin,
                       &h_tile_slots);
  const size_t Phs = static_cast<size_t>(g.H) * shf::fast_pitch(g);
  const size_t y_elems = Phs * static_cast<size_t>(std::max(plan.y_planes, 1));
  const size_t partial_elems = static_cast<size_t>(std::max(plan.nslots, 1)) * g.H * shf::fast_tile(g);
  float2 *Y = nullptr, *partial = nullptr;
  shf::WorkItem* items = nullptr;
  int *cta_begin = nullptr, *tile_begin = nullptr, *tile_slots = nullptr;
  auto release = [&]() {
    cudaFree(Y);
    cudaFree(partial);
    cudaFree(items);
    cudaFree(cta_begin);
    cudaFree(tile_begin);
    cudaFree(tile_slots);
  };
  int rc;
  if ((rc = dev_alloc(&Y, y_elems, "Y")) || (rc = dev_alloc(&partial, partial_elems, "partial")) ||
      (rc = dev_alloc(&items, h_items.size(), "work items")) ||
      (rc = dev_alloc(&cta_begin, h_cta_begin.size(), "work ranges")) ||
      (rc = dev_alloc(&tile_begin, h_tile_begin.size(), "tile_begin")) ||
      (rc = dev_alloc(&tile_slots, h_tile_slots.size(), "tile_slots"))) {
    release();
    return rc;
  }
  cudaError_t e = cudaMemcpy(items, h_items.data(), sizeof(shf::WorkItem) * h_items.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(cta_begin, h_cta_begin.data(), sizeof(int) * h_cta_begin.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(tile_begin, h_tile_begin.data(), sizeof(int) * h_tile_begin.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(tile_slots, h_tile_slots.data(), sizeof(int) * h_tile_slots.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st->stream);  // the old buffers may still be in use
  if (e != cudaSuccess) {
    release();
    return fail(SHF_ERR_CUDA, std::string("install_fast_plan: ") + cudaGetErrorString(e));
  }
  drop_graphs(st);
  cudaFree(st->Y);
  cudaFree(st->partial);
  cudaFree(st->d_items);
  cudaFree(st->d_cta_begin);
  cudaFree(st->d_tile_begin);
  cudaFree(st->d_tile_slots);
  st->Y = Y;
  st->partial = partial;
  st->d_items = items;
  st->d_cta_begin = cta_begin;
  st->d_tile_begin = tile_begin;
  st->d_tile_slots = tile_slots;
  plan.items = items;
  plan.cta_begin = cta_begin;
  plan.tile_begin = tile_begin;
  plan.tile_slots = tile_slots;
  st->plan = plan;
  return SHF_OK;
}

// Filter groups as the general-path kernels use them: groups of ceil(eta/G)
// filters, no group empty.
int normalise_groups(int eta, int G) {
  if (G < 1) G = 1;
  if (G > eta) G = eta;
  const int fg = (eta + G - 1) / G;
  return (eta + fg - 1) / fg;
}

// General path: tile shape (TC, RB) and filter groups; reallocates the
// partial sums.  Synchronises the state's stream.
int install_generic_plan(seg_state* st, int TC, int RB, int groups) {
  int dev = 0, optin = 0;
  SHF_CK(cudaGetDevice(&dev));
  SHF_CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  Geo g = st->g;
  if (!shf::set_generic_tiles(&g, TC, RB, st->K, optin))
    return fail(SHF_ERR_ARG, "tile shape not supported for this image size");
  groups = normalise_groups(g.eta, groups);
  float2* partial = nullptr;
  int rc = dev_alloc(&partial, st->Ph() * st->K * static_cast<size_t>(groups), "partial");
  if (rc) return rc;
  cudaError_t e = cudaStreamSynchronize(st->stream);
  if (e != cudaSuccess) {
    cudaFree(partial);
    return fail(SHF_ERR_CUDA, std::string("install_generic_plan: ") + cudaGetErrorString(e));
  }
  drop_graphs(st);
  cudaFree(st->partial);
  st->partial = partial;
  st->g = g;
  st->groups = groups;
  return SHF_OK;
}

int energy_of_w(seg_state* st, double* out_host) {
  const Geo& g = st->g;
  const size_t P = st->P();
  const float scale = 1.f / (static_cast<float>(g.H) * g.W);
  // <w, s>
  SHF_CK(shf::launch_dot(st->w, st->s, static_cast<long>(P * st->K), st->red + 2, 512, st->red, st->stream));
  // sum_f Lambda_f ||(S w)_f||_1: row-forward of w, fan-out over all filters,
  // l1 of the row-inverse; the spectra of all K*eta planes go to stream-ordered
  // temporaries (the state's scratch holds one wave of filters on the fast path).
  const size_t ph = st->Ph();
  float2* tmp = nullptr;
  SHF_CK(cudaMallocAsync(reinterpret_cast<void**>(&tmp), sizeof(float2) * ph * st->K * (1 + g.eta), st->stream));
  float2* Uw = tmp;
  float2* Yw = tmp + ph * st->K;
  cudaError_t e = shf::run_row_r2c(g, st->w, Uw, st->K, 1.f, st->stream);
  if (e == cudaSuccess) e = shf::run_col_fan(g, Uw, Yw, st->K, st->groups, st->stream);
  int nb = 0;
  if (e == cudaSuccess) e = shf::run_row_l1(g, Yw, st->lam, st->K * g.eta, scale, st->red + 2 + 512, &nb, st->stream);
  cudaError_t e2 = cudaFreeAsync(tmp, st->stream);
  SHF_CK(e);
  SHF_CK(e2);
  SHF_CK(shf::launch_sum_partials(st->red + 2 + 512, nb, st->red + 1, st->stream));
  double h[2];
  SHF_CK(cudaMemcpyAsync(h, st->red, sizeof(h), cudaMemcpyDeviceToHost, st->stream));
  SHF_CK(cudaStreamSynchronize(st->stream));
  *out_host = h[0] + h[1];
  return SHF_OK;
}

int residual_uw(seg_state* st, double* out_host) {
  const size_t n = st->P() * st->K;
  SHF_CK(shf::launch_sqdiff(st->u, st->w, static_cast<long>(n), st->red + 2, 512, st->red, st->stream));
  double h = 0;
  SHF_CK(cudaMemcpyAsync(&h, st->red, sizeof(double), cudaMemcpyDeviceToHost, st->stream));
  SHF_CK(cudaStreamSynchronize(st->stream));
  *out_host = std::sqrt(h / static_cast<double>(n));
  return SHF_OK;
}

int copy_out(seg_state* st, void* dst, const void* src, size_t bytes, int to_host) {
  SHF_CK(cudaMemcpyAsync(dst, src, bytes, to_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st->stream));
  if (to_host) SHF_CK(cudaStreamSynchronize(st->stream));
  return SHF_OK;
}

int copy_in(seg_state* st, void* dst, const void* src, size_t bytes, int from_host) {
  SHF_CK(cudaMemcpyAsync(dst, src, bytes, from_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st->stream));
  if (from_host) SHF_CK(cudaStreamSynchronize(st->stream));
  return SHF_OK;
}

}  // namespace

int seg_admm_init(const shf_bank* b, const float* f, int C, const float* codebook, int K, const seg_params* p,
                  void* stream, seg_state** out) {
  if (!out) return fail(SHF_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!b || !f || !codebook || !p || !p->Lambda) return fail(SHF_ERR_ARG, "seg_admm_init: NULL argument");
  if (K < 2 || K > shf::kMaxK) return fail(SHF_ERR_ARG, "K must be in [2, 16]");
  if (C != 1 && C != 3) return fail(SHF_ERR_ARG, "C must be 1 or 3");
  if (p->J != b->g.J) return fail(SHF_ERR_STATE, "params->J differs from the bank's J");
  if (!(p->gamma > 0.f) || !std::isfinite(p->gamma)) return fail(SHF_ERR_ARG, "gamma must be positive and finite");
  if (!aligned8(f)) return fail(SHF_ERR_ARG, "f must be 8-byte aligned");
  for (int i = 0; i < K * C; ++i)
    if (!std::isfinite(codebook[i])) return fail(SHF_ERR_NONFINITE, "codebook contains NaN or Inf");
  for (int j = 0; j <= p->J; ++j)
    if (!std::isfinite(p->Lambda[j]) || p->Lambda[j] < 0.f)
      return fail(SHF_ERR_ARG, "Lambda must be finite and non-negative");
  auto* st = new seg_state();
  st->bank = b;
  st->g = b->g;
  st->K = K;
  st->C = C;
  st->gamma = p->gamma;
  st->Lambda.assign(p->Lambda, p->Lambda + p->J + 1);
  st->codebook.assign(codebook, codebook + K * C);
  st->max_iters = p->max_iters;
  st->tol = p->tol;
  st->check_every = p->check_every > 0 ? p->check_every : 1;
  if (stream) {
    st->stream = static_cast<cudaStream_t>(stream);
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&st->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete st;
      return fail(SHF_ERR_CUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
    }
    st->own_stream = true;
  }
  const Geo& g = st->g;
  const size_t P = st->P(), Ph = st->Ph();
  st->groups = shf::default_groups(g, K);
  st->fast = shf::fast_path_ok(g);
  st->fast_ustep = shf::fast_ustep_ok(g, K);
  // the fast path's work list is built from the filters' column ranges
  if (st->fast) {
    st->ranges_host.resize(g.eta);
    cudaError_t e = cudaMemcpy(st->ranges_host.data(), g.ranges, sizeof(int2) * g.eta, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
      free_state(st);
      return fail(SHF_ERR_CUDA, std::string("seg_admm_init: ") + cudaGetErrorString(e));
    }
  }
  const int l1_blocks = ((g.H + g.RB - 1) / g.RB) * K * g.eta;
  st->red_len = 2 + 512 + l1_blocks;
  int rc;
  if ((rc = dev_alloc(&st->f, P * C, "f")) || (rc = dev_alloc(&st->s, P * K, "s")) ||
      (rc = dev_alloc(&st->bv, P * K * g.eta, "b_v")) || (rc = dev_alloc(&st->w, P * K, "w")) ||
      (rc = dev_alloc(&st->bw, P * K, "b_w")) || (rc = dev_alloc(&st->u, P * K, "u")) ||
      (rc = dev_alloc(&st->stv, P * K, "stv")) || (rc = dev_alloc(&st->Ur, Ph * K, "Ur")) ||
      (rc = dev_alloc(&st->T, Ph * K, "T")) ||
      (st->fast && (rc = dev_alloc(&st->uhat, static_cast<size_t>(g.H) * shf::fast_pitch(g) * K, "uhat"))) ||
      // coefficient spectra of the whole label set and one partial sum per
      // filter group on the general path (the fast path's come with its plan)
      (!st->fast && (rc = dev_alloc(&st->Y, Ph * K * g.eta, "Y"))) ||
      (!st->fast && (rc = dev_alloc(&st->partial, Ph * K * static_cast<size_t>(st->groups), "partial"))) ||
      (st->fast && (rc = install_fast_plan(st, shf::kDefaultWaveMiB, 0))) ||
      (rc = dev_alloc(&st->thr, g.eta, "thr")) || (rc = dev_alloc(&st->lam, g.eta, "lam")) ||
      (rc = dev_alloc(&st->gap, P, "gap")) || (rc = dev_alloc(&st->labels, P, "labels")) ||
      (rc = dev_alloc(&st->flag, 1, "flag")) || (rc = dev_alloc(&st->red, st->red_len, "red"))) {
    free_state(st);
    return rc;
  }
  std::vector<shf::FilterDesc> d(g.eta);
  shf::filter_descs(g.J, d.data());
  std::vector<float> thr(g.eta), lam(g.eta);
  for (int i = 0; i < g.eta; ++i) {
    lam[i] = d[i].kind == 0 ? st->Lambda[0] : st->Lambda[d[i].j + 1];
    thr[i] = st->gamma * lam[i];
  }
  cudaError_t e = cudaMemcpyAsync(st->thr, thr.data(), sizeof(float) * g.eta, cudaMemcpyHostToDevice, st->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(st->lam, lam.data(), sizeof(float) * g.eta, cudaMemcpyHostToDevice, st->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(st->f, f, sizeof(float) * P * C, cudaMemcpyDeviceToDevice, st->stream);
  if (e != cudaSuccess) {
    free_state(st);
    return fail(SHF_ERR_CUDA, std::string("seg_admm_init: ") + cudaGetErrorString(e));
  }
  rc = restart(st, codebook);  // synchronises: thr/lam host vectors stay valid until here
  if (rc) {
    free_state(st);
    return rc;
  }
  *out = st;
  return SHF_OK;
}

int seg_admm_reset(seg_state* st, const float* f, int f_on_host) {
  if (!st || !f) return fail(SHF_ERR_ARG, "seg_admm_reset: NULL argument");
  if (!f_on_host && !aligned8(f)) return fail(SHF_ERR_ARG, "f must be 8-byte aligned");
  SHF_CK(cudaMemcpyAsync(st->f, f, sizeof(float) * st->P() * st->C,
                         f_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st->stream));
  return restart(st, st->codebook.data());
}

int seg_admm_step(seg_state* st, int n) {
  if (!st || n < 0) return fail(SHF_ERR_ARG, "seg_admm_step: bad argument");
  if (n == 0) return SHF_OK;
  if (!st->graph_tried) try_capture(st);
  // the last iteration of the call records the per-kernel timing events
  for (int i = 0; i < n; ++i) {
    const bool timed = i == n - 1 && !st->untimed;
    if (st->exec) {
      SHF_CK(cudaGraphLaunch(timed && st->exec_timed ? st->exec_timed : st->exec, st->stream));
    } else {
      SHF_CK(enqueue_iteration(st, timed));
    }
  }
  st->iter += n;
  return SHF_OK;
}

int seg_admm_get_plan(const seg_state* st, seg_plan* out) {
  if (!st || !out) return fail(SHF_ERR_ARG, "seg_admm_get_plan: NULL argument");
  out->fast = st->fast ? 1 : 0;
  out->wave_mib = st->fast ? st->plan.wave_mib : 0;
  out->col_ctas_per_sm = st->fast ? st->plan.col_ctas_per_sm : 0;
  out->tile_cols = st->fast ? 0 : st->g.TC;
  out->tile_rows = st->fast ? 0 : st->g.RB;
  out->groups = st->fast ? 0 : st->groups;
  out->us_per_iter = 0.f;
  out->row_kernel = st->fast ? st->plan.row_kernel : 0;
  out->col_kernel = st->fast ? st->plan.col_kernel : 0;
  out->serial = st->fast ? st->plan.serial : 0;
  out->sms = st->fast ? st->plan.sms : 0;
  return SHF_OK;
}

int seg_admm_set_plan(seg_state* st, const seg_plan* p) {
  if (!st || !p) return fail(SHF_ERR_ARG, "seg_admm_set_plan: NULL argument");
  if (st->fast) {
    if (p->col_ctas_per_sm < 0 || p->col_ctas_per_sm > 32 || p->wave_mib < 1 || p->wave_mib > 4096)
      return fail(SHF_ERR_ARG, "seg_admm_set_plan: col_ctas_per_sm must be in [0, 32] and wave_mib in [1, 4096]");
    if (!shf::fast_row_kernel_ok(st->g, p->row_kernel) || !shf::fast_col_kernel_ok(st->g, p->col_kernel))
      return fail(SHF_ERR_ARG, "seg_admm_set_plan: row_kernel or col_kernel not available at this size");
    if (p->serial != 0 && p->serial != 1) return fail(SHF_ERR_ARG, "seg_admm_set_plan: serial must be 0 or 1");
    if (p->sms < 0 || p->sms > 65536) return fail(SHF_ERR_ARG, "seg_admm_set_plan: sms must be in [0, 65536]");
    if (p->col_ctas_per_sm == st->plan.col_ctas_per_sm && p->wave_mib == st->plan.wave_mib &&
        p->row_kernel == st->plan.row_kernel && p->col_kernel == st->plan.col_kernel && p->sms == st->plan.sms) {
      if (p->serial != st->plan.serial) {  // same buffers, other launches: capture the graphs again
        st->plan.serial = p->serial;
        drop_graphs(st);
      }
      return SHF_OK;
    }
    return install_fast_plan(st, p->wave_mib, p->col_ctas_per_sm, p->row_kernel, p->col_kernel, p->serial, p->sms);
  }
  if (p->tile_cols < 1 || p->tile_rows < 1 || p->groups < 1)
    return fail(SHF_ERR_ARG, "seg_admm_set_plan: tile_cols, tile_rows and groups must be positive");
  if (p->tile_cols == st->g.TC && p->tile_rows == st->g.RB && normalise_groups(st->g.eta, p->groups) == st->groups)
    return SHF_OK;
  return install_generic_plan(st, p->tile_cols, p->tile_rows, p->groups);
}

}  // extern "C"

namespace {

// Mean time (microseconds) of one iteration over `iters` replays, after one
// warm-up iteration that also captures the graphs.
// Average time of `iters` iterations of the plain graph (without the event
// nodes of the timed iteration, which cost differently per plan).
int time_iterations(seg_state* st, int iters, float* us) {
  st->untimed = true;
  struct Restore {
    seg_state* st;
    ~Restore() { st->untimed = false; }
  } restore{st};
  int rc = seg_admm_step(st, 1);
  if (rc) return rc;
  cudaEvent_t a = nullptr, b = nullptr;
  SHF_CK(cudaEventCreate(&a));
  cudaError_t e = cudaEventCreate(&b);
  if (e == cudaSuccess) e = cudaEventRecord(a, st->stream);
  if (e == cudaSuccess) rc = seg_admm_step(st, iters);
  if (e == cudaSuccess && !rc) e = cudaEventRecord(b, st->stream);
  if (e == cudaSuccess && !rc) e = cudaEventSynchronize(b);
  float ms = 0.f;
  if (e == cudaSuccess && !rc) e = cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (rc) return rc;
  SHF_CK(e);
  *us = 1000.f * ms / static_cast<float>(iters);
  return SHF_OK;
}

// Candidate plans around the current one, for coordinate-wise search: stage 0
// varies the first parameter, stage 1 the second, stage 2 the third, each
// around the best found so far.
std::vector<seg_plan> plan_candidates(const seg_state* st, const seg_plan& base, int stage) {
  std::vector<seg_plan> out;
  const Geo& g = st->g;
  if (st->fast) {
    if (stage == 0) {
      // wave budgets that give distinct waves (filters per wave of one label,
      // or labels per wave)
      std::vector<int> seen;
      for (int mib : {16, 32, 64, 96, 128, 192, 256, 384}) {
        const int w = shf::fast_wave(g, mib), nl = shf::fast_wave_labels(g, mib, st->K);
        const int sig = nl > 1 ? -nl : (g.eta + w - 1) / w;
        if (std::find(seen.begin(), seen.end(), sig) != seen.end()) continue;
        seen.push_back(sig);
        seg_plan p = base;
        p.wave_mib = mib;
        out.push_back(p);
      }
    } else if (stage == 2) {
      // the FFT kernel of the forward v-step: 8 or 16 values per thread, one
      // row or a pair of rows per group, or 12 / 20 / 32 values per thread
      // (odd factor 3 or 5, or 1024 = 32 x 32); each with the iteration's
      // launches overlapped (programmatic dependent launch) and serial
      for (int rk : {shf::kRow8, shf::kRow16, shf::kRowPair, shf::kRowV}) {
        if (!shf::fast_row_kernel_ok(g, rk)) continue;
        for (int serial : {0, 1}) {  // with and without programmatic dependent launch
          seg_plan p = base;
          p.row_kernel = rk;
          p.serial = serial;
          out.push_back(p);
        }
      }
    } else if (stage == 3) {
      // the FFT kernel of the fan and the gather: 8 or 16 values per thread
      for (int ck : {shf::kCol8, shf::kCol16, shf::kColV}) {
        if (!shf::fast_col_kernel_ok(g, ck)) continue;
        seg_plan p = base;
        p.col_kernel = ck;
        out.push_back(p);
      }
    } else if (stage == 1) {
      // resident column CTAs per SM: every count up to what fits (0 = all)
      const int fit = shf::fast_col_ctas(g, 0, base.col_kernel) / std::max(1, shf::fast_col_ctas(g, 1, base.col_kernel));
      for (int c = 1; c < fit; ++c) {
        seg_plan p = base;
        p.col_ctas_per_sm = c;
        out.push_back(p);
      }
      seg_plan p = base;
      p.col_ctas_per_sm = 0;
      out.push_back(p);
    }
    return out;
  }
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return out;
  if (stage == 0) {
    std::vector<int> seen;
    for (int G : {base.groups / 2, base.groups, 2 * base.groups, 4 * base.groups}) {
      const int n = normalise_groups(g.eta, G);
      if (std::find(seen.begin(), seen.end(), n) != seen.end()) continue;
      seen.push_back(n);
      seg_plan p = base;
      p.groups = n;
      out.push_back(p);
    }
  } else if (stage == 1 || stage == 2) {
    const int vals1[] = {4, 8, 16, 32};
    const int vals2[] = {base.tile_rows / 2, base.tile_rows, 2 * base.tile_rows};
    const int* vals = stage == 1 ? vals1 : vals2;
    const int nv = stage == 1 ? 4 : 3;
    for (int i = 0; i < nv; ++i) {
      seg_plan p = base;
      (stage == 1 ? p.tile_cols : p.tile_rows) = vals[i];
      Geo t = g;
      if (!shf::set_generic_tiles(&t, p.tile_cols, p.tile_rows, st->K, optin)) continue;
      out.push_back(p);
    }
  }
  return out;
}

// A copy of a state's iterate (b_v, w, b_w, u and the u-spectra) and
// iteration count, taken on the state's stream before trial iterations and
// put back after them.
struct IterateCopy {
  seg_state* st = nullptr;
  float* buf = nullptr;
  long long iter0 = 0;

  // SHF_ERR_OOM when there is no memory for the copy
  int save(seg_state* s) {
    st = s;
    iter0 = s->iter;
    const size_t KP = s->P() * s->K, NC = KP * s->g.eta, TH = s->Ph() * s->K;
    if (cudaMallocAsync(reinterpret_cast<void**>(&buf), sizeof(float) * (NC + 3 * KP + 2 * TH), s->stream) !=
        cudaSuccess) {
      cudaGetLastError();
      buf = nullptr;
      return fail(SHF_ERR_OOM, "no memory to save the iterate for the tuning trials");
    }
    return copy(true) == cudaSuccess ? SHF_OK : fail(SHF_ERR_CUDA, "saving the iterate failed");
  }
  // copies the iterate back, frees the copy and synchronises the stream
  cudaError_t restore() {
    if (!buf) return cudaSuccess;
    cudaError_t e = copy(false);
    cudaError_t e2 = cudaFreeAsync(buf, st->stream);
    cudaError_t e3 = cudaStreamSynchronize(st->stream);
    buf = nullptr;
    st->iter = iter0;
    return e != cudaSuccess ? e : (e2 != cudaSuccess ? e2 : e3);
  }

 private:
  cudaError_t copy(bool save) {
    const size_t KP = st->P() * st->K, NC = KP * st->g.eta, TH = st->Ph() * st->K;
    struct Piece {
      void* p;
      size_t bytes;
    };
    const Piece pieces[] = {{st->bv, sizeof(float) * NC},
                            {st->w, sizeof(float) * KP},
                            {st->bw, sizeof(float) * KP},
                            {st->u, sizeof(float) * KP},
                            {st->T, sizeof(float2) * TH}};
    char* q = reinterpret_cast<char*>(buf);
    cudaError_t e = cudaSuccess;
    for (const Piece& pc : pieces) {
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(save ? q : pc.p, save ? pc.p : q, pc.bytes, cudaMemcpyDeviceToDevice, st->stream);
      q += pc.bytes;
    }
    return e;
  }
};

}  // namespace

extern "C" {

int seg_admm_tune(seg_state* st, int iters, seg_plan* best_out) {
  if (!st || iters < 1) return fail(SHF_ERR_ARG, "seg_admm_tune: bad argument");
  // the iterate is saved and restored around the trial iterations
  IterateCopy snap;
  int rc0 = snap.save(st);
  if (rc0) {
    snap.restore();
    return rc0;
  }
  seg_plan best;
  seg_admm_get_plan(st, &best);
  best.us_per_iter = INFINITY;
  int rc = SHF_OK;
  for (int stage = 0; stage < 4 && !rc; ++stage) {
    const seg_plan base = best;
    for (const seg_plan& cand : plan_candidates(st, base, stage)) {
      int r = seg_admm_set_plan(st, &cand);
      if (r == SHF_ERR_OOM || r == SHF_ERR_ARG) continue;  // not feasible here: skip
      if (r) {
        rc = r;
        break;
      }
      // the better of two timings: plans a few percent apart must not swap
      // places on one noisy trial
      float us = 0.f, us2 = 0.f;
      r = time_iterations(st, iters, &us);
      if (!r) r = time_iterations(st, iters, &us2);
      if (r) {
        rc = r;
        break;
      }
      us = std::min(us, us2);
      if (us < best.us_per_iter) {
        best = cand;
        best.us_per_iter = us;
      }
    }
  }
  if (!rc) rc = seg_admm_set_plan(st, &best);
  const cudaError_t e = snap.restore();
  if (rc) return rc;
  if (e != cudaSuccess) return fail(SHF_ERR_CUDA, "seg_admm_tune: restoring the iterate failed");
  if (best_out) *best_out = best;
  return SHF_OK;
}

int seg_admm_solve(seg_state* st, int* iters_done, float* final_residual) {
  if (!st) return fail(SHF_ERR_ARG, "state is NULL");
  double res = INFINITY;
  int done = 0;
  while (done < st->max_iters) {
    const int n = std::min(st->check_every, st->max_iters - done);
    int rc = seg_admm_step(st, n);
    if (rc) return rc;
    done += n;
    rc = residual_uw(st, &res);
    if (rc) return rc;
    if (res < st->tol) break;
  }
  if (iters_done) *iters_done = done;
  if (final_residual) *final_residual = static_cast<float>(res);
  return SHF_OK;
}

int seg_admm_get(seg_state* st, int what, void* dst, int on_host) {
  if (!st || !dst) return fail(SHF_ERR_ARG, "seg_admm_get: NULL argument");
  const Geo& g = st->g;
  const size_t P = st->P(), KP = P * st->K;
  switch (what) {
    case SEG_U: return copy_out(st, dst, st->u, sizeof(float) * KP, on_host);
    case SEG_W: return copy_out(st, dst, st->w, sizeof(float) * KP, on_host);
    case SEG_BW: return copy_out(st, dst, st->bw, sizeof(float) * KP, on_host);
    case SEG_BV: return copy_out(st, dst, st->bv, sizeof(float) * KP * g.eta, on_host);
    case SEG_S: return copy_out(st, dst, st->s, sizeof(float) * KP, on_host);
    case SEG_STV:
      SHF_CK(shf::run_row_c2r(g, st->T, st->stv, st->K, 1.f / (static_cast<float>(g.H) * g.W), st->stream));
      return copy_out(st, dst, st->stv, sizeof(float) * KP, on_host);
    case SEG_LABELS:
    case SEG_GAP:
      SHF_CK(shf::launch_labels(st->w, st->K, static_cast<int>(P), st->labels, st->gap, st->stream));
      if (what == SEG_LABELS) return copy_out(st, dst, st->labels, sizeof(int) * P, on_host);
      return copy_out(st, dst, st->gap, sizeof(float) * P, on_host);
    case SEG_ENERGY: {
      double e = 0;
      int rc = energy_of_w(st, &e);
      if (rc) return rc;
      if (on_host) {
        *static_cast<double*>(dst) = e;
        return SHF_OK;
      }
      SHF_CK(cudaMemcpy(dst, &e, sizeof(double), cudaMemcpyHostToDevice));
      return SHF_OK;
    }
    case SEG_ITER:
      if (!on_host) return fail(SHF_ERR_ARG, "SEG_ITER is host only");
      *static_cast<int*>(dst) = static_cast<int>(st->iter);
      return SHF_OK;
    default: return fail(SHF_ERR_ARG, "unknown selector");
  }
}

int seg_admm_set(seg_state* st, int what, const void* src, int on_host) {
  if (!st || !src) return fail(SHF_ERR_ARG, "seg_admm_set: NULL argument");
  const Geo& g = st->g;
  const size_t P = st->P(), KP = P * st->K;
  switch (what) {
    case SEG_W: return copy_in(st, st->w, src, sizeof(float) * KP, on_host);
    case SEG_BW: return copy_in(st, st->bw, src, sizeof(float) * KP, on_host);
    case SEG_BV: return copy_in(st, st->bv, src, sizeof(float) * KP * g.eta, on_host);
    case SEG_STV: {
      int rc = copy_in(st, st->stv, src, sizeof(float) * KP, on_host);
      if (rc) return rc;
      // T = H * row-forward(stv), so that the u-step's 1/(HW) row-inverse returns stv.
      SHF_CK(shf::run_row_r2c(g, st->stv, st->T, st->K, static_cast<float>(g.H), st->stream));
      return SHF_OK;
    }
    case SEG_V: {
      float* d = nullptr;
      SHF_CK(cudaMallocAsync(reinterpret_cast<void**>(&d), sizeof(float) * KP * g.eta, st->stream));
      cudaError_t e = cudaMemcpyAsync(d, src, sizeof(float) * KP * g.eta,
                                      on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st->stream);
      if (e == cudaSuccess) e = shf::launch_sub(d, st->bv, d, static_cast<long>(KP * g.eta), st->stream);
      if (e == cudaSuccess) e = synthesis_spectrum(g, d, st->K, st->T, st->stream);
      cudaError_t e2 = cudaFreeAsync(d, st->stream);
      if (e == cudaSuccess) e = e2;
      if (e == cudaSuccess && on_host) e = cudaStreamSynchronize(st->stream);
      if (e != cudaSuccess) return fail(SHF_ERR_CUDA, std::string("seg_admm_set(SEG_V): ") + cudaGetErrorString(e));
      return SHF_OK;
    }
    default: return fail(SHF_ERR_ARG, "selector cannot be set");
  }
}

namespace {
struct CkptHeader {
  char magic[8];
  int32_t H, W, K, J, eta, C;
  int64_t iter;
  float gamma;
  float Lambda[shf::kMaxJ + 1];
};
}  // namespace

int seg_admm_save(seg_state* st, const char* path) {
  if (!st || !path) return fail(SHF_ERR_ARG, "seg_admm_save: NULL argument");
  const Geo& g = st->g;
  const size_t KP = st->P() * st->K;
  CkptHeader h{};
  std::memcpy(h.magic, "SHFCKPT1", 8);
  h.H = g.H;
  h.W = g.W;
  h.K = st->K;
  h.J = g.J;
  h.eta = g.eta;
  h.C = st->C;
  h.iter = st->iter;
  h.gamma = st->gamma;
  for (int j = 0; j <= g.J; ++j) h.Lambda[j] = st->Lambda[j];
  std::vector<float> buf(KP * g.eta);
  FILE* fp = std::fopen(path, "wb");
  if (!fp) return fail(SHF_ERR_IO, std::string("cannot open ") + path);
  bool ok = std::fwrite(&h, sizeof(h), 1, fp) == 1;
  // the carried synthesis spectrum T, raw, so that a resumed run continues bit for bit
  const size_t nT = 2 * st->Ph() * st->K;
  std::vector<float> tbuf(nT);
  int rc0 = copy_out(st, tbuf.data(), st->T, sizeof(float) * nT, 1);
  if (rc0) {
    std::fclose(fp);
    return rc0;
  }
  ok = ok && std::fwrite(tbuf.data(), sizeof(float), nT, fp) == nT;
  const int parts[] = {SEG_BV, SEG_W, SEG_BW, SEG_S, SEG_U};
  for (int what : parts) {
    const size_t n = what == SEG_BV ? KP * g.eta : KP;
    int rc = seg_admm_get(st, what, buf.data(), 1);
    if (rc) {
      std::fclose(fp);
      return rc;
    }
    ok = ok && std::fwrite(buf.data(), sizeof(float), n, fp) == n;
  }
  ok = (std::fclose(fp) == 0) && ok;
  return ok ? SHF_OK : fail(SHF_ERR_IO, std::string("write failed: ") + path);
}

int seg_admm_load(seg_state* st, const char* path) {
  if (!st || !path) return fail(SHF_ERR_ARG, "seg_admm_load: NULL argument");
  const Geo& g = st->g;
  const size_t KP = st->P() * st->K;
  FILE* fp = std::fopen(path, "rb");
  if (!fp) return fail(SHF_ERR_IO, std::string("cannot open ") + path);
  CkptHeader h{};
  if (std::fread(&h, sizeof(h), 1, fp) != 1 || std::memcmp(h.magic, "SHFCKPT1", 8) != 0) {
    std::fclose(fp);
    return fail(SHF_ERR_IO, "not a checkpoint file");
  }
  if (h.H != g.H || h.W != g.W || h.K != st->K || h.J != g.J) {
    std::fclose(fp);
    return fail(SHF_ERR_STATE, "checkpoint sizes differ from the state's");
  }
  std::vector<float> buf(KP * g.eta);
  const size_t nT = 2 * st->Ph() * st->K;
  std::vector<float> tbuf(nT);
  if (std::fread(tbuf.data(), sizeof(float), nT, fp) != nT) {
    std::fclose(fp);
    return fail(SHF_ERR_IO, "truncated checkpoint");
  }
  int rc0 = copy_in(st, st->T, tbuf.data(), sizeof(float) * nT, 1);
  if (rc0) {
    std::fclose(fp);
    return rc0;
  }
  const int parts[] = {SEG_BV, SEG_W, SEG_BW};
  for (int what : parts) {
    const size_t n = what == SEG_BV ? KP * g.eta : KP;
    if (std::fread(buf.data(), sizeof(float), n, fp) != n) {
      std::fclose(fp);
      return fail(SHF_ERR_IO, "truncated checkpoint");
    }
    int rc = seg_admm_set(st, what, buf.data(), 1);
    if (rc) {
      std::fclose(fp);
      return rc;
    }
  }
  // s and u
  for (float* dstp : {st->s, st->u}) {
    if (std::fread(buf.data(), sizeof(float), KP, fp) != KP) {
      std::fclose(fp);
      return fail(SHF_ERR_IO, "truncated checkpoint");
    }
    int rc = copy_in(st, dstp, buf.data(), sizeof(float) * KP, 1);
    if (rc) {
      std::fclose(fp);
      return rc;
    }
  }
  std::fclose(fp);
  st->iter = h.iter;
  return SHF_OK;
}

}  // extern "C"

namespace {

// Layout of the reverse sweep's temporaries in st->un_mem (byte offsets, each
// region on a 256-byte boundary: the fast kernels copy rows of bvbar and of
// the codes with 16-byte asynchronous copies).
struct UnLayout {
  size_t tpart, tbar, cbpart, cbout;      // doubles
  size_t Uw, Tt;                          // float2 [K][H][Wh]
  size_t bvbar, dbar, Qbar, wbar, bwbar, sbar, gwbar, stv, fbar, grec, wrec;  // floats
  size_t code;                            // bytes
  size_t total;
};

UnLayout un_layout(const seg_state* st, int ck) {
  const Geo& g = st->g;
  const int K = st->K, C = st->C, eta = g.eta;
  const size_t P = st->P(), Ph = st->Ph(), KP = P * K, NC = KP * eta;
  const bool fast = st->fast;
  const size_t nblk = static_cast<size_t>(shf::adj_part_blocks());
  UnLayout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off = (off + bytes + 255) & ~static_cast<size_t>(255);
    return at;
  };
  L.tpart = take(sizeof(double) * K * eta * (fast ? static_cast<size_t>(g.H) : nblk));
  L.tbar = take(sizeof(double) * eta);
  L.cbpart = take(sizeof(double) * K * C * nblk);
  L.cbout = take(sizeof(double) * K * C);
  L.Uw = take(sizeof(float2) * Ph * K);
  L.Tt = take(sizeof(float2) * Ph * K);
  L.bvbar = take(sizeof(float) * NC);
  L.dbar = fast ? 0 : take(sizeof(float) * NC);
  L.Qbar = take(sizeof(float) * KP);
  L.wbar = take(sizeof(float) * KP);
  L.bwbar = take(sizeof(float) * KP);
  L.sbar = take(sizeof(float) * KP);
  L.gwbar = take(sizeof(float) * KP);
  L.stv = take(sizeof(float) * KP);
  L.fbar = take(sizeof(float) * P * C);
  L.grec = fast ? 0 : take(sizeof(float) * NC * ck);
  L.wrec = take(sizeof(float) * KP * ck);
  L.code = fast ? take(NC * ck) : 0;
  L.total = off;
  return L;
}

// T iterations from the zero state, keeping (b_v, w, b_w, T) before every
// ckpt-th iteration.
cudaError_t enqueue_unrolled_fwd(seg_state* st, int T, int ck) {
  const size_t P = st->P(), Ph = st->Ph(), KP = P * st->K, NC = KP * st->g.eta;
  cudaStream_t s = st->stream;
  cudaError_t e = cudaSuccess;
  auto ok = [&](cudaError_t x) {
    if (e == cudaSuccess) e = x;
  };
  ok(cudaMemsetAsync(st->bv, 0, sizeof(float) * NC, s));
  ok(cudaMemsetAsync(st->w, 0, sizeof(float) * KP, s));
  ok(cudaMemsetAsync(st->bw, 0, sizeof(float) * KP, s));
  ok(cudaMemsetAsync(st->u, 0, sizeof(float) * KP, s));
  ok(cudaMemsetAsync(st->T, 0, sizeof(float2) * Ph * st->K, s));
  for (int i = 0; i < T && e == cudaSuccess; ++i) {
    if (i % ck == 0) {
      const int c = i / ck;
      ok(cudaMemcpyAsync(st->ck_bv[c], st->bv, sizeof(float) * NC, cudaMemcpyDeviceToDevice, s));
      ok(cudaMemcpyAsync(st->ck_w[c], st->w, sizeof(float) * KP, cudaMemcpyDeviceToDevice, s));
      ok(cudaMemcpyAsync(st->ck_bw[c], st->bw, sizeof(float) * KP, cudaMemcpyDeviceToDevice, s));
      ok(cudaMemcpyAsync(st->ck_T[c], st->T, sizeof(float2) * Ph * st->K, cudaMemcpyDeviceToDevice, s));
    }
    ok(st->fast ? enqueue_iteration(st, false) : enqueue_generic_iteration(st, nullptr));
  }
  return e;
}

// The reverse sweep, from wbar (already holding dL/dw) to sbar, fbar, tbar
// and cbout in st->un_mem.
cudaError_t enqueue_unrolled_bwd(seg_state* st, const UnLayout& U) {
  const Geo& g = st->g;
  const int K = st->K, C = st->C, eta = g.eta, T = st->un_T, ck = st->un_ck;
  const size_t P = st->P(), Ph = st->Ph(), KP = P * K, NC = KP * eta;
  const float scale = 1.f / (static_cast<float>(g.H) * g.W);
  cudaStream_t s = st->stream;
  const bool fast = st->fast;
  char* m = st->un_mem;
  double* tpart = reinterpret_cast<double*>(m + U.tpart);
  double* tbar = reinterpret_cast<double*>(m + U.tbar);
  double* cbpart = reinterpret_cast<double*>(m + U.cbpart);
  double* cbout = reinterpret_cast<double*>(m + U.cbout);
  float2* Uw = reinterpret_cast<float2*>(m + U.Uw);
  float2* Tt = reinterpret_cast<float2*>(m + U.Tt);
  auto F = [&](size_t o) { return reinterpret_cast<float*>(m + o); };
  float *bvbar = F(U.bvbar), *dbar = fast ? nullptr : F(U.dbar), *Qbar = F(U.Qbar), *wbar = F(U.wbar),
        *bwbar = F(U.bwbar), *sbar = F(U.sbar), *gwbar = F(U.gwbar), *stv = F(U.stv), *fbar = F(U.fbar),
        *grec = fast ? nullptr : F(U.grec), *wrec = F(U.wrec);
  signed char* crec = fast ? reinterpret_cast<signed char*>(m + U.code) : nullptr;
  cudaError_t e = cudaSuccess;
  auto ok = [&](cudaError_t x) {
    if (e == cudaSuccess) e = x;
    return e == cudaSuccess;
  };
  ok(cudaMemsetAsync(bvbar, 0, sizeof(float) * NC, s));
  ok(cudaMemsetAsync(Qbar, 0, sizeof(float) * KP, s));
  ok(cudaMemsetAsync(bwbar, 0, sizeof(float) * KP, s));
  ok(cudaMemsetAsync(sbar, 0, sizeof(float) * KP, s));
  ok(cudaMemsetAsync(tbar, 0, sizeof(double) * eta, s));
  const int nseg = (T + ck - 1) / ck;
  for (int seg = nseg - 1; seg >= 0 && e == cudaSuccess; --seg) {
    const int n = std::min(ck, T - seg * ck);
    ok(cudaMemcpyAsync(st->bv, st->ck_bv[seg], sizeof(float) * NC, cudaMemcpyDeviceToDevice, s));
    ok(cudaMemcpyAsync(st->w, st->ck_w[seg], sizeof(float) * KP, cudaMemcpyDeviceToDevice, s));
    ok(cudaMemcpyAsync(st->bw, st->ck_bw[seg], sizeof(float) * KP, cudaMemcpyDeviceToDevice, s));
    ok(cudaMemcpyAsync(st->T, st->ck_T[seg], sizeof(float2) * Ph * K, cudaMemcpyDeviceToDevice, s));
    for (int i = 0; i < n && e == cudaSuccess; ++i) {  // recompute the segment, recording g (or its codes) and w'
      if (fast)
        ok(enqueue_iteration(st, false, crec + static_cast<size_t>(i) * NC));
      else
        ok(enqueue_generic_iteration(st, grec + static_cast<size_t>(i) * NC));
      ok(cudaMemcpyAsync(wrec + static_cast<size_t>(i) * KP, st->w, sizeof(float) * KP, cudaMemcpyDeviceToDevice, s));
    }
    for (int i = n - 1; i >= 0 && e == cudaSuccess; --i) {
      ok(shf::launch_adj_proj(wrec + static_cast<size_t>(i) * KP, wbar, bwbar, gwbar, K, static_cast<int>(P), s));
      if (fast) {
        // S Qbar, the v-step adjoint and S^T bvbar, fused per wave of filters
        ok(shf::run_row_r2c(g, Qbar, Uw, K, 1.f, s));
        ok(shf::run_fast_adjoint_body(g, st->plan, Uw, st->uhat, st->Y, bvbar, st->thr, st->partial, Tt, K, scale,
                                      crec + static_cast<size_t>(i) * NC, tpart, s));
        ok(shf::launch_adj_tsum_rows(tpart, K, eta, g.H, tbar, s));
      } else {
        // dbar = S Qbar
        ok(shf::run_row_r2c(g, Qbar, Uw, K, 1.f, s));
        ok(shf::run_col_fan(g, Uw, st->un_Y, K, st->groups, s));
        ok(shf::run_row_c2r(g, st->un_Y, dbar, K * eta, scale, s));
        ok(shf::launch_adj_shrink(grec + static_cast<size_t>(i) * NC, dbar, bvbar, st->thr, K, eta,
                                  static_cast<long>(P), tpart, tbar, s));
        // stv = S^T bvbar
        ok(shf::run_row_r2c(g, bvbar, st->un_Y, K * eta, 1.f, s));
        ok(shf::run_col_gather(g, st->un_Y, st->un_partial, K, st->un_groups, s));
        ok(shf::run_col_reduce_inv(g, st->un_partial, Tt, K, st->un_groups, s));
      }
      ok(shf::run_row_c2r(g, Tt, stv, K, scale, s));
      ok(shf::launch_adj_u(gwbar, stv, Qbar, wbar, bwbar, sbar, st->gamma, static_cast<long>(KP), s));
    }
  }
  ok(shf::adj_codebook(sbar, st->f, st->codebook.data(), K, C, static_cast<long>(P), cbpart, cbout, fbar, s));
  return e;
}

}  // namespace

extern "C" {

int seg_admm_unrolled_fwd(seg_state* st, int T, int ckpt_every) {
  if (!st || T < 1 || ckpt_every < 1) return fail(SHF_ERR_ARG, "seg_admm_unrolled_fwd: bad argument");
  const Geo& g = st->g;
  const size_t P = st->P(), Ph = st->Ph(), KP = P * st->K, NC = KP * g.eta;
  int rc;
  // the general path keeps the spectra of every filter; the fast path
  // iterates with its own wave scratch
  if (!st->fast && !st->un_Y) {
    if ((rc = dev_alloc(&st->un_Y, Ph * st->K * g.eta, "unrolled scratch")) ||
        (rc = dev_alloc(&st->un_partial, Ph * st->K * st->groups, "unrolled partials")))
      return rc;
    st->un_groups = st->groups;
  }
  const int nseg = (T + ckpt_every - 1) / ckpt_every;
  while (static_cast<int>(st->ck_bv.size()) < nseg) {
    float *bv = nullptr, *w = nullptr, *bw = nullptr;
    float2* Tt = nullptr;
    if ((rc = dev_alloc(&bv, NC, "checkpoint")) || (rc = dev_alloc(&w, KP, "checkpoint")) ||
        (rc = dev_alloc(&bw, KP, "checkpoint")) || (rc = dev_alloc(&Tt, Ph * st->K, "checkpoint"))) {
      cudaFree(bv);
      cudaFree(w);
      cudaFree(bw);
      cudaFree(Tt);
      return rc;
    }
    st->ck_bv.push_back(bv);
    st->ck_w.push_back(w);
    st->ck_bw.push_back(bw);
    st->ck_T.push_back(Tt);
  }
  // one graph per (T, ckpt), replayed by later calls
  if (!(st->un_fwd_exec && st->un_fwd_key[0] == T && st->un_fwd_key[1] == ckpt_every)) {
    if (st->un_fwd_exec) cudaGraphExecDestroy(st->un_fwd_exec);
    st->un_fwd_exec = capture_work(st, [&]() { return enqueue_unrolled_fwd(st, T, ckpt_every); });
    st->un_fwd_key[0] = T;
    st->un_fwd_key[1] = ckpt_every;
  }
  if (st->un_fwd_exec)
    SHF_CK(cudaGraphLaunch(st->un_fwd_exec, st->stream));
  else
    SHF_CK(enqueue_unrolled_fwd(st, T, ckpt_every));
  st->iter = T;
  st->un_T = T;
  st->un_ck = ckpt_every;
  return SHF_OK;
}

int seg_admm_unrolled_bwd_enqueue(seg_state* st, const float* dL_dw) {
  if (!st || !dL_dw) return fail(SHF_ERR_ARG, "seg_admm_unrolled_bwd_enqueue: NULL argument");
  if (st->un_T < 1) return fail(SHF_ERR_STATE, "seg_admm_unrolled_fwd has not run");
  const size_t KP = st->P() * st->K;
  cudaStream_t s = st->stream;
  const UnLayout U = un_layout(st, st->un_ck);
  if (st->un_mem_bytes < U.total) {
    SHF_CK(cudaStreamSynchronize(s));
    if (st->un_bwd_exec) cudaGraphExecDestroy(st->un_bwd_exec);
    st->un_bwd_exec = nullptr;
    cudaFree(st->un_mem);
    st->un_mem = nullptr;
    st->un_mem_bytes = 0;
    int rc = dev_alloc(&st->un_mem, U.total, "reverse-sweep scratch");
    if (rc) return rc;
    st->un_mem_bytes = U.total;
  }
  SHF_CK(cudaMemcpyAsync(st->un_mem + U.wbar, dL_dw, sizeof(float) * KP, cudaMemcpyDeviceToDevice, s));
  // one graph per (T, ckpt), replayed by later calls
  if (!(st->un_bwd_exec && st->un_bwd_key[0] == st->un_T && st->un_bwd_key[1] == st->un_ck)) {
    if (st->un_bwd_exec) cudaGraphExecDestroy(st->un_bwd_exec);
    st->un_bwd_exec = capture_work(st, [&]() { return enqueue_unrolled_bwd(st, U); });
    st->un_bwd_key[0] = st->un_T;
    st->un_bwd_key[1] = st->un_ck;
  }
  SHF_CK(st->un_bwd_exec ? cudaGraphLaunch(st->un_bwd_exec, s) : enqueue_unrolled_bwd(st, U));
  st->un_bwd_pending = true;
  return SHF_OK;
}

int seg_admm_unrolled_grads(seg_state* st, float* dL_dcodebook, float* dL_dLambda, float* dL_df, float* dL_ds) {
  if (!st || !dL_dcodebook || !dL_dLambda) return fail(SHF_ERR_ARG, "seg_admm_unrolled_grads: NULL argument");
  if (!st->un_bwd_pending) return fail(SHF_ERR_STATE, "no reverse sweep has been enqueued");
  const Geo& g = st->g;
  const int K = st->K, C = st->C, eta = g.eta;
  const size_t P = st->P(), KP = P * K;
  cudaStream_t s = st->stream;
  const UnLayout U = un_layout(st, st->un_ck);
  char* m = st->un_mem;
  cudaError_t e = cudaSuccess;
  auto ok = [&](cudaError_t x) {
    if (e == cudaSuccess) e = x;
  };
  if (dL_df) ok(cudaMemcpyAsync(dL_df, m + U.fbar, sizeof(float) * P * C, cudaMemcpyDeviceToDevice, s));
  if (dL_ds) ok(cudaMemcpyAsync(dL_ds, m + U.sbar, sizeof(float) * KP, cudaMemcpyDeviceToDevice, s));
  std::vector<double> th(eta), cb(static_cast<size_t>(K) * C);
  ok(cudaMemcpyAsync(th.data(), m + U.tbar, sizeof(double) * eta, cudaMemcpyDeviceToHost, s));
  ok(cudaMemcpyAsync(cb.data(), m + U.cbout, sizeof(double) * K * C, cudaMemcpyDeviceToHost, s));
  ok(cudaStreamSynchronize(s));
  if (e != cudaSuccess) return fail(SHF_ERR_CUDA, std::string("seg_admm_unrolled_grads: ") + cudaGetErrorString(e));
  std::vector<shf::FilterDesc> d(eta);
  shf::filter_descs(g.J, d.data());
  std::vector<double> lam(g.J + 1, 0.0);
  for (int f = 0; f < eta; ++f) lam[d[f].kind == 0 ? 0 : d[f].j + 1] += st->gamma * th[f];
  for (int j = 0; j <= g.J; ++j) dL_dLambda[j] = static_cast<float>(lam[j]);
  for (int i = 0; i < K * C; ++i) dL_dcodebook[i] = static_cast<float>(cb[i]);
  return SHF_OK;
}

int seg_admm_unrolled_bwd(seg_state* st, const float* dL_dw, float* dL_dcodebook, float* dL_dLambda, float* dL_df,
                          float* dL_ds) {
  if (!st || !dL_dw || !dL_dcodebook || !dL_dLambda) return fail(SHF_ERR_ARG, "seg_admm_unrolled_bwd: NULL argument");
  int rc = seg_admm_unrolled_bwd_enqueue(st, dL_dw);
  if (rc) return rc;
  return seg_admm_unrolled_grads(st, dL_dcodebook, dL_dLambda, dL_df, dL_ds);
}

int seg_admm_kernel_times(seg_state* st, float* ms, int* launches, int* nk) {
  if (!st || !ms) return fail(SHF_ERR_ARG, "seg_admm_kernel_times: NULL argument");
  if (st->iter == 0 || st->nmarks < 2) return fail(SHF_ERR_STATE, "no iteration has run yet");
  if (!st->marks_ok) return fail(SHF_ERR_STATE, "iteration has more launches than timing marks");
  for (int k = 0; k < shf::kNumKinds; ++k) {
    ms[k] = 0.f;
    if (launches) launches[k] = 0;
  }
  SHF_CK(cudaEventSynchronize(st->ev[st->nmarks - 1]));
  for (int i = 0; i + 1 < st->nmarks; ++i) {
    float t = 0.f;
    SHF_CK(cudaEventElapsedTime(&t, st->ev[i], st->ev[i + 1]));
    ms[st->kinds[i]] += t;
    if (launches) ++launches[st->kinds[i]];
  }
  if (nk) *nk = shf::kNumKinds;
  return SHF_OK;
}

const char* seg_admm_kernel_name(int i) {
  static const char* names[] = {"row_ustep", "col_fwd", "col_fan", "row_shrink", "col_gather", "col_reduce_inv"};
  return (i >= 0 && i < shf::kNumKinds) ? names[i] : "";
}

// ---------------------------------------------------------------------------
// Batches
// ---------------------------------------------------------------------------
}  // extern "C"

struct seg_batch {
  std::vector<shf_bank*> banks;
  std::vector<seg_state*> states;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> joins;
  cudaGraphExec_t exec = nullptr;
  bool graph_tried = false;
  int lanes = 0;  // chains of images run side by side (0: one image per chain)
};

namespace {

void drop_batch_graphs(seg_batch* b) {
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
  b->graph_tried = false;
}

int tune_batch_layout(seg_batch* b, int iters);

void free_batch(seg_batch* b) {
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
  for (seg_state* s : b->states)
    if (s) s->batch = nullptr;
  for (seg_state* s : b->states)
    if (s) seg_admm_destroy(s);
  for (shf_bank* k : b->banks)
    if (k) shfilters_destroy(k);
  if (b->fork) cudaEventDestroy(b->fork);
  for (cudaEvent_t e : b->joins)
    if (e) cudaEventDestroy(e);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

// Forks from the batch stream, enqueues one iteration of every image on its
// own stream and joins back.  With b->lanes = L in [1, n) the images form L
// chains that run side by side: in decreasing order of their work (H W K eta)
// each image joins the chain with the least work so far and starts after the
// chain's previous image; with 0 (or L >= n) every image is a chain of its own.
cudaError_t enqueue_batch_iteration(seg_batch* b) {
  const int n = static_cast<int>(b->states.size());
  const int nl = b->lanes > 0 && b->lanes < n ? b->lanes : n;
  auto work = [&](int i) {
    const seg_state* s = b->states[i];
    return static_cast<double>(s->P()) * s->K * s->g.eta;
  };
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  if (nl < n) std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return work(x) > work(y); });
  std::vector<double> load(nl, 0.0);
  std::vector<int> last(nl, -1);  // the chain's latest image
  cudaError_t e = cudaEventRecord(b->fork, b->stream);
  for (int k = 0; k < n && e == cudaSuccess; ++k) {
    const int i = order[k];
    int l = nl < n ? 0 : k;
    if (nl < n)
      for (int c = 1; c < nl; ++c)
        if (load[c] < load[l]) l = c;
    load[l] += work(i);
    seg_state* st = b->states[i];
    e = cudaStreamWaitEvent(st->stream, last[l] < 0 ? b->fork : b->joins[last[l]], 0);
    if (e == cudaSuccess) e = enqueue_iteration(st, false);
    if (e == cudaSuccess) e = cudaEventRecord(b->joins[i], st->stream);
    last[l] = i;
  }
  for (int l = 0; l < nl && e == cudaSuccess; ++l)
    if (last[l] >= 0) e = cudaStreamWaitEvent(b->stream, b->joins[last[l]], 0);
  return e;
}

}  // namespace

extern "C" {

int seg_admm_batch_init(int n, const int* H, const int* W, const int* C, const int* K, const float* const* f,
                        const float* const* codebooks, const seg_params* params, void* stream, seg_batch** out) {
  if (!out) return fail(SHF_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (n < 1 || !H || !W || !C || !K || !f || !codebooks || !params)
    return fail(SHF_ERR_ARG, "seg_admm_batch_init: bad argument");
  auto* b = new seg_batch();
  if (stream) {
    b->stream = static_cast<cudaStream_t>(stream);
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete b;
      return fail(SHF_ERR_CUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
    }
    b->own_stream = true;
  }
  cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    free_batch(b);
    return fail(SHF_ERR_CUDA, std::string("cudaEventCreate: ") + cudaGetErrorString(e));
  }
  b->joins.assign(n, nullptr);
  for (int i = 0; i < n; ++i) {
    e = cudaEventCreateWithFlags(&b->joins[i], cudaEventDisableTiming);
    if (e != cudaSuccess) {
      free_batch(b);
      return fail(SHF_ERR_CUDA, std::string("cudaEventCreate: ") + cudaGetErrorString(e));
    }
  }
  b->states.assign(n, nullptr);
  for (int i = 0; i < n; ++i) {
    shf_bank* bank = nullptr;
    for (shf_bank* k : b->banks)
      if (k->g.H == H[i] && k->g.W == W[i] && k->g.J == params[i].J) bank = k;
    if (!bank) {
      int rc = shfilters_build(H[i], W[i], params[i].J, b->stream, &bank);
      if (rc) {
        const std::string m = g_err;
        free_batch(b);
        return fail(rc, "image " + std::to_string(i) + ": " + m);
      }
      b->banks.push_back(bank);
    }
    int rc = seg_admm_init(bank, f[i], C[i], codebooks[i], K[i], &params[i], nullptr, &b->states[i]);
    if (rc) {
      const std::string m = g_err;
      free_batch(b);
      return fail(rc, "image " + std::to_string(i) + ": " + m);
    }
    b->states[i]->batch = b;
  }
  *out = b;
  return SHF_OK;
}

int seg_admm_batch_step(seg_batch* b, int n) {
  if (!b || n < 0) return fail(SHF_ERR_ARG, "seg_admm_batch_step: bad argument");
  if (n == 0) return SHF_OK;
  if (!b->graph_tried) {
    b->graph_tried = true;
    cudaGraph_t graph = nullptr;
    if (b->stream && cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      cudaError_t e = enqueue_batch_iteration(b);
      cudaError_t e2 = cudaStreamEndCapture(b->stream, &graph);
      if (e == cudaSuccess && e2 == cudaSuccess && graph &&
          cudaGraphInstantiate(&b->exec, graph, 0) != cudaSuccess)
        b->exec = nullptr;
      if (graph) cudaGraphDestroy(graph);
    }
    cudaGetLastError();
  }
  for (int i = 0; i < n; ++i) {
    if (b->exec) {
      SHF_CK(cudaGraphLaunch(b->exec, b->stream));
    } else {
      SHF_CK(enqueue_batch_iteration(b));
    }
  }
  for (seg_state* st : b->states) st->iter += n;
  return SHF_OK;
}

int seg_admm_batch_set_lanes(seg_batch* b, int lanes) {
  if (!b || lanes < 0) return fail(SHF_ERR_ARG, "seg_admm_batch_set_lanes: bad argument");
  if (lanes != b->lanes) {
    b->lanes = lanes;
    drop_batch_graphs(b);
  }
  return SHF_OK;
}

int seg_admm_batch_get_lanes(const seg_batch* b, int* lanes) {
  if (!b || !lanes) return fail(SHF_ERR_ARG, "seg_admm_batch_get_lanes: NULL argument");
  *lanes = b->lanes;
  return SHF_OK;
}

int seg_admm_batch_image(seg_batch* b, int i, seg_state** out) {
  if (!b || !out || i < 0 || i >= static_cast<int>(b->states.size()))
    return fail(SHF_ERR_ARG, "seg_admm_batch_image: bad argument");
  *out = b->states[i];
  return SHF_OK;
}

}  // extern "C"

namespace {

// Mean time (microseconds) of one batch iteration over `iters` replays of the
// batch's graph, after one that also captures it.
int time_batch_iterations(seg_batch* b, int iters, float* us) {
  int rc = seg_admm_batch_step(b, 1);
  if (rc) return rc;
  cudaEvent_t a = nullptr, c = nullptr;
  SHF_CK(cudaEventCreate(&a));
  cudaError_t e = cudaEventCreate(&c);
  if (e == cudaSuccess) e = cudaEventRecord(a, b->stream);
  if (e == cudaSuccess) rc = seg_admm_batch_step(b, iters);
  if (e == cudaSuccess && !rc) e = cudaEventRecord(c, b->stream);
  if (e == cudaSuccess && !rc) e = cudaEventSynchronize(c);
  float ms = 0.f;
  if (e == cudaSuccess && !rc) e = cudaEventElapsedTime(&ms, a, c);
  cudaEventDestroy(a);
  if (c) cudaEventDestroy(c);
  if (rc) return rc;
  SHF_CK(e);
  *us = 1000.f * ms / static_cast<float>(iters);
  return SHF_OK;
}

// The fast images' fan, v-step and gather grids sized for `sms` SMs (0: all).
int set_batch_share(seg_batch* b, int sms) {
  for (seg_state* st : b->states) {
    if (!st->fast) continue;
    seg_plan p;
    seg_admm_get_plan(st, &p);
    p.sms = sms;
    const int rc = seg_admm_set_plan(st, &p);
    if (rc) return rc;
  }
  return SHF_OK;
}

// Batch-wide stages of the tuner, timed on the batch's graph (each candidate
// twice, the better time kept; the iterates saved before and restored after,
// or the stages skipped without memory for the copies): first the number of
// image chains (one image per chain, or 1 to 4 chains), then every fast
// image's persistent grids sized for all SMs or for a half, a third or a
// quarter of them.
int tune_batch_layout(seg_batch* b, int iters) {
  const int n = static_cast<int>(b->states.size());
  if (n < 2) return SHF_OK;
  int nfast = 0;
  for (seg_state* st : b->states) nfast += st->fast ? 1 : 0;
  int dev = 0, nsm = 0;
  SHF_CK(cudaGetDevice(&dev));
  SHF_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  std::vector<IterateCopy> snaps(b->states.size());
  int rc = SHF_OK;
  for (size_t i = 0; i < b->states.size() && !rc; ++i) rc = snaps[i].save(b->states[i]);
  for (seg_state* st : b->states) cudaStreamSynchronize(st->stream);  // copies before the batch's streams
  auto timed = [&](float* best_us) {
    float us = INFINITY;
    for (int t = 0; t < 2 && !rc; ++t) {
      float u = 0.f;
      rc = time_batch_iterations(b, iters, &u);
      us = std::min(us, u);
    }
    const bool better = !rc && us < *best_us;
    if (better) *best_us = us;
    return better;
  };
  int best_lanes = b->lanes, best_share = 0;
  if (!rc) {
    float best_us = INFINITY;
    for (int lanes : {0, 1, 2, 3, 4}) {
      if (lanes >= n) continue;
      b->lanes = lanes;
      drop_batch_graphs(b);
      if (timed(&best_us)) best_lanes = lanes;
      if (rc) break;
    }
    b->lanes = best_lanes;
    drop_batch_graphs(b);
    best_us = INFINITY;
    for (int share : {0, nsm / 2, nsm / 3, nsm / 4}) {
      if (rc || nfast == 0 || (share > 0 && share < 8)) continue;
      rc = set_batch_share(b, share);
      if (!rc && timed(&best_us)) best_share = share;
    }
  }
  const bool skipped = rc == SHF_ERR_OOM;
  if (skipped) rc = SHF_OK;
  b->lanes = best_lanes;
  drop_batch_graphs(b);
  if (!rc) rc = set_batch_share(b, best_share);
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (IterateCopy& sn : snaps)
    if (sn.restore() != cudaSuccess && !rc) rc = fail(SHF_ERR_CUDA, "seg_admm_batch_tune: restoring an iterate failed");
  return rc;
}

}  // namespace

extern "C" {

int seg_admm_batch_tune(seg_batch* b, int iters) {
  if (!b || iters < 1) return fail(SHF_ERR_ARG, "seg_admm_batch_tune: bad argument");
  // every image back on grids for all SMs before its shape is tuned alone
  for (seg_state* st : b->states) {
    if (!st->fast || st->plan.sms == 0) continue;
    seg_plan p;
    seg_admm_get_plan(st, &p);
    p.sms = 0;
    const int rc = seg_admm_set_plan(st, &p);
    if (rc) return rc;
  }
  // one tuning run per distinct problem shape; the other images take its plan
  struct Key {
    int fast, H, W, J, K;
    bool operator==(const Key& o) const {
      return fast == o.fast && H == o.H && W == o.W && J == o.J && K == o.K;
    }
  };
  std::vector<std::pair<Key, seg_plan>> done;
  for (seg_state* st : b->states) {
    const Key k{st->fast ? 1 : 0, st->g.H, st->g.W, st->g.J, st->K};
    auto it = std::find_if(done.begin(), done.end(), [&](const std::pair<Key, seg_plan>& d) { return d.first == k; });
    int rc;
    if (it == done.end()) {
      seg_plan p;
      rc = seg_admm_tune(st, iters, &p);
      if (!rc) done.emplace_back(k, p);
    } else {
      rc = seg_admm_set_plan(st, &it->second);
    }
    if (rc) return rc;
  }
  drop_batch_graphs(b);
  return tune_batch_layout(b, iters);
}

int seg_admm_batch_sync(seg_batch* b) {
  if (!b) return fail(SHF_ERR_ARG, "batch is NULL");
  SHF_CK(cudaStreamSynchronize(b->stream));
  return SHF_OK;
}

int seg_admm_batch_destroy(seg_batch* b) {
  if (!b) return SHF_OK;
  free_batch(b);
  return SHF_OK;
}

int seg_admm_sync(seg_state* st) {
  if (!st) return fail(SHF_ERR_ARG, "state is NULL");
  SHF_CK(cudaStreamSynchronize(st->stream));
  return SHF_OK;
}

int seg_admm_destroy(seg_state* st) {
  if (!st) return SHF_OK;
  cudaStreamSynchronize(st->stream);
  free_state(st);
  return SHF_OK;
}

}  // extern "C"

// Fast path of an ADMM iteration (Sec. 3 of Haeuser & Steidl) for image sizes
// whose height H and half width L = W/2 are register-FFT lengths R 2^a
// (R in {1, 3, 5}, 8 <= R 2^a <= 1024): host-side work plan and launch
// sequence.  The kernels are in shf_fast_col.cu and shf_fast_row.cu.
//
// One iteration:
//   row_ustep       u/w-step and b_w update, row spectra of u -> Ur
//   col_fwd         Ur -> uhat, the full 2-D spectrum of u, once per label;
//   per wave of (label, filter) pairs (the filters [f0, f0 + nf) of one label,
//   or whole labels [l0, l0 + nl) when their spectra fit the wave budget):
//     col_fan         Y_v = column-inverse(W_f * uhat_k) for (k, f) in the wave
//     row_shrink      row-inverse, g = b_v + S u, b_v <- clip(g), d = soft(g) -
//                     clip(g) (= v - b_v), row-forward of d, in place in Y_v
//     col_gather      partial slots += W_f * column-forward(Y_v)
//   col_reduce      T_k = column-inverse(sum of the partial slots)
// The coefficient spectra of one wave stay in (or, for two 512^2 labels, just
// exceed) L2 between the three kernels; b_v is streamed with evict-first
// hints.  Kernel variants by size: the v-step on pairs of rows (half widths 64,
// 128), radix-16 rows (256 .. 1024) or 8-value rows (other widths); the fan
// and gather with radix-16 columns at heights 512 and 1024.
#include <algorithm>

#include "shf_fast.h"

namespace shf {

int fast_pitch(const Geo& g) { return (g.Wh + 7) & ~7; }

bool fast_path_ok(const Geo& g) { return reg::supported_col(g.H) && reg::supported(g.L); }

int fast_tile(const Geo& g) { return reg::col_batch(g.H); }

bool fast_ustep_ok(const Geo& g, int K) {
  if (!fast_path_ok(g) || K > 8) return false;
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return false;
  const size_t need = fast::ustep_smem_bytes(g.L, K);
  return need > 0 && need <= static_cast<size_t>(optin);
}

cudaError_t prepare_fast_kernels() {
  cudaError_t e = fast::prepare_col_kernels();
  if (e == cudaSuccess) e = fast::prepare_row_kernels();
  return e;
}

cudaError_t run_fast_ustep(const Geo& g, const float2* T, const float* s, float* w, float* bw, float* u, float2* Ur,
                           int K, float gamma, float scale, cudaStream_t st) {
  return fast::row_ustep(g, T, s, w, bw, u, Ur, K, gamma, scale, st);
}

namespace {
// coefficient-spectra planes that fit the wave budget
int wave_planes(const Geo& g, int wave_mib) {
  const size_t plane = sizeof(float2) * static_cast<size_t>(g.H) * fast_pitch(g);
  const size_t w = (static_cast<size_t>(wave_mib) << 20) / plane;
  return static_cast<int>(std::max<size_t>(1, std::min<size_t>(w, 1 << 20)));
}
}  // namespace

int fast_wave(const Geo& g, int wave_mib) {
  // filters per wave of one label: keep the wave's coefficient spectra near
  // wave_mib MiB, with the waves of a label balanced
  const int w = std::min(wave_planes(g, wave_mib), g.eta);
  const int nw = (g.eta + w - 1) / w;
  return (g.eta + nw - 1) / nw;
}

int fast_wave_labels(const Geo& g, int wave_mib, int K) {
  // whole labels per wave when at least two labels' spectra fit, balanced
  // over the label groups
  const int nl = std::min(K, wave_planes(g, wave_mib) / g.eta);
  if (nl < 2) return 1;
  const int ng = (K + nl - 1) / nl;
  return (K + ng - 1) / ng;
}

namespace {
int sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  return sms;
}
}  // namespace

// SMs a plan's persistent grids are sized for
int sms_for(int sms) {
  const int n = sm_count();
  return sms > 0 && sms < n ? sms : n;
}

int fast_col_ctas(const Geo& g, int per_sm, int col_kernel, int sms) {
  const int fit = fast::col_ctas_per_sm(g.H, col_kernel);
  if (fit < 1) return 0;
  const int k = (per_sm <= 0 || per_sm > fit) ? fit : per_sm;
  return k * sms_for(sms);
}

int fast_row_ctas(const Geo& g, int row_kernel, int sms) {
  return fast::row_ctas_per_sm(g.L, 0, row_kernel) * sms_for(sms);
}

int fast_fan_ctas(const Geo& g, int col_kernel, int sms) { return fast::fan_ctas_per_sm(g.H, col_kernel) * sms_for(sms); }

bool fast_row_kernel_ok(const Geo& g, int row_kernel) { return fast::row_kernel_ok(g.L, row_kernel); }

bool fast_col_kernel_ok(const Geo& g, int col_kernel) { return fast::col_kernel_ok(g.H, col_kernel); }

void build_fast_plan(const Geo& g, const int2* ranges, int K, FastPlan* plan, std::vector<WorkItem>* items,
                     std::vector<int>* cta_begin, std::vector<int>* tile_begin, std::vector<int>* tile_slots) {
  const int tw = fast_tile(g), ntiles = (g.Wh + tw - 1) / tw;
  const int ctas = plan->col_ctas > 0 ? plan->col_ctas : 1;
  items->clear();
  cta_begin->clear();
  plan->wave_l0.clear();
  plan->wave_nl.clear();
  plan->wave_f0.clear();
  plan->wave_nf.clear();
  plan->wave_cta0.clear();
  plan->wave_fcta0.clear();
  plan->y_planes = 0;
  // the waves: label groups of whole labels, or per label the filter waves
  const int nl = fast_wave_labels(g, plan->wave_mib, K);
  if (nl > 1) {
    for (int l0 = 0; l0 < K; l0 += nl) {
      plan->wave_l0.push_back(l0);
      plan->wave_nl.push_back(std::min(nl, K - l0));
      plan->wave_f0.push_back(0);
      plan->wave_nf.push_back(g.eta);
    }
  } else {
    const int wave = fast_wave(g, plan->wave_mib);
    for (int k = 0; k < K; ++k)
      for (int f0 = 0; f0 < g.eta; f0 += wave) {
        plan->wave_l0.push_back(k);
        plan->wave_nl.push_back(1);
        plan->wave_f0.push_back(f0);
        plan->wave_nf.push_back(std::min(wave, g.eta - f0));
      }
  }
  std::vector<std::vector<int>> per_tile(static_cast<size_t>(K) * ntiles);
  int slot = 0;
  for (size_t w = 0; w < plan->wave_f0.size(); ++w) {
    const int l0 = plan->wave_l0[w], wl = plan->wave_nl[w], f0 = plan->wave_f0[w], nf = plan->wave_nf[w];
    plan->y_planes = std::max(plan->y_planes, wl * nf);
    // this wave's (label, tile, filter) triples in that order
    const size_t first = items->size();
    for (int k = l0; k < l0 + wl; ++k)
      for (int t = 0; t < ntiles; ++t)
        for (int f = f0; f < f0 + nf; ++f) {
          const int2 r = ranges[f];
          if (r.x <= r.y && t >= r.x / tw && t <= r.y / tw) items->push_back(WorkItem{t, f, 0, k});
        }
    const long n = static_cast<long>(items->size() - first);
    const int G = static_cast<int>(std::min<long>(ctas, n));
    plan->wave_cta0.push_back(static_cast<int>(cta_begin->size()) - static_cast<int>(plan->wave_cta0.size()));
    for (int c = 0; c <= G; ++c) cta_begin->push_back(static_cast<int>(first + (G > 0 ? n * c / G : 0)));
    // one partial slot per run of one (label, tile) inside a CTA's range
    for (int c = 0; c < G; ++c) {
      const long b = n * c / G, e = n * (c + 1) / G;
      for (long i = b; i < e; ++i) {
        WorkItem& it = (*items)[first + i];
        const WorkItem* prev = i == b ? nullptr : &(*items)[first + i - 1];
        if (!prev || prev->tile != it.tile || prev->label != it.label)
          per_tile[static_cast<size_t>(it.label) * ntiles + it.tile].push_back(slot++);
        it.slot = slot - 1;
      }
    }
  }
  plan->wave_cta0.push_back(static_cast<int>(cta_begin->size()) - static_cast<int>(plan->wave_cta0.size()));
  // the fan's ranges over the same items, for its own number of CTAs
  {
    const int fctas = plan->fan_ctas > 0 ? plan->fan_ctas : ctas;
    size_t first = 0;
    for (size_t w = 0; w < plan->wave_f0.size(); ++w) {
      const int c0 = plan->wave_cta0[w] + static_cast<int>(w), c1 = plan->wave_cta0[w + 1] + static_cast<int>(w) + 1;
      const long n = (*cta_begin)[c1 - 1] - (*cta_begin)[c0];  // the wave's items
      first = static_cast<size_t>((*cta_begin)[c0]);
      const int G = static_cast<int>(std::min<long>(fctas, n));
      plan->wave_fcta0.push_back(static_cast<int>(cta_begin->size()) - static_cast<int>(plan->wave_fcta0.size()));
      for (int c = 0; c <= G; ++c) cta_begin->push_back(static_cast<int>(first + (G > 0 ? n * c / G : 0)));
    }
    plan->wave_fcta0.push_back(static_cast<int>(cta_begin->size()) - static_cast<int>(plan->wave_fcta0.size()));
  }
  plan->nslots = slot;
  tile_begin->assign(1, 0);
  tile_slots->clear();
  for (const auto& lst : per_tile) {
    for (int sl : lst) tile_slots->push_back(sl);
    tile_begin->push_back(static_cast<int>(tile_slots->size()));
  }
  if (items->empty()) items->push_back(WorkItem{0, 0, 0, 0});  // keep the device arrays non-empty
  if (tile_slots->empty()) tile_slots->push_back(0);
}

cudaError_t run_fast_iteration_body(const Geo& g, const FastPlan& plan, const float2* Ur, float2* uhat, float2* Y,
                                    float* bv, const float* thr, float2* partial, float2* T, int K, float scale,
                                    cudaStream_t st, const LaunchHook& hook, signed char* code) {
  const int Whp = fast_pitch(g);
  const int nw = static_cast<int>(plan.wave_f0.size());
  const int rpc = fast::row_groups_per_cta(g.L, 0, plan.row_kernel);
  hook.mark(kKindColFwd);
  cudaError_t e = fast::col_fwd(g, Ur, uhat, K, Whp, st);
  for (int w = 0; w < nw && e == cudaSuccess; ++w) {
    const fast::Wave wv{plan.wave_l0[w], plan.wave_f0[w], plan.wave_nf[w], plan.wave_nl[w] * plan.wave_nf[w]};
    const int c0 = plan.wave_cta0[w], nc = plan.wave_cta0[w + 1] - c0;
    const int* cb = plan.cta_begin + c0 + w;  // each wave's ranges end with one extra entry
    const int f0c = plan.wave_fcta0[w], nfc = plan.wave_fcta0[w + 1] - f0c;
    const int* fcb = plan.cta_begin + f0c + w;
    if (nfc > 0) {
      hook.mark(kKindFan);
      e = fast::col_fan(g, nfc, uhat, plan.items, fcb, Y, Whp, wv, plan.col_kernel, st);
    }
    hook.mark(kKindShrink);
    const int groups = (wv.nv * g.H + rpc - 1) / rpc;
    const int ctas = std::min(groups, std::max(plan.row_ctas, 1));
    if (e == cudaSuccess) e = fast::row_shrink(g, ctas, Y, bv, thr, Whp, wv, scale, code, plan.row_kernel, st);
    if (nc > 0 && e == cudaSuccess) {
      hook.mark(kKindGather);
      e = fast::col_gather(g, nc, Y, plan.items, cb, partial, Whp, wv, plan.col_kernel, st);
    }
  }
  hook.mark(kKindReduce);
  if (e == cudaSuccess) e = fast::col_reduce(g, partial, plan.tile_begin, plan.tile_slots, T, K, st);
  return e;
}

cudaError_t run_fast_adjoint_body(const Geo& g, const FastPlan& plan, const float2* Qr, float2* uhat, float2* Y,
                                  float* bvbar, const float* thr, float2* partial, float2* Tbar, int K, float scale,
                                  const signed char* code, double* tpart, cudaStream_t st) {
  const PdlScope pdl(!plan.serial);
  const int Whp = fast_pitch(g);
  const int nw = static_cast<int>(plan.wave_f0.size());
  const int rpc = fast::row_groups_per_cta(g.L, 1);
  const int actas = fast::row_ctas_per_sm(g.L, 1) * sm_count();
  cudaError_t e = fast::col_fwd(g, Qr, uhat, K, Whp, st);
  for (int w = 0; w < nw && e == cudaSuccess; ++w) {
    const fast::Wave wv{plan.wave_l0[w], plan.wave_f0[w], plan.wave_nf[w], plan.wave_nl[w] * plan.wave_nf[w]};
    const int c0 = plan.wave_cta0[w], nc = plan.wave_cta0[w + 1] - c0;
    const int* cb = plan.cta_begin + c0 + w;
    const int f0c = plan.wave_fcta0[w], nfc = plan.wave_fcta0[w + 1] - f0c;
    const int* fcb = plan.cta_begin + f0c + w;
    if (nfc > 0) e = fast::col_fan(g, nfc, uhat, plan.items, fcb, Y, Whp, wv, plan.col_kernel, st);
    const int groups = (wv.nv * g.H + rpc - 1) / rpc;
    const int ctas = std::min(groups, std::max(actas, 1));
    if (e == cudaSuccess) e = fast::row_adjoint(g, ctas, Y, bvbar, thr, Whp, wv, scale, code, tpart, st);
    if (nc > 0 && e == cudaSuccess) e = fast::col_gather(g, nc, Y, plan.items, cb, partial, Whp, wv, plan.col_kernel, st);
  }
  if (e == cudaSuccess) e = fast::col_reduce(g, partial, plan.tile_begin, plan.tile_slots, Tbar, K, st);
  return e;
}

}  // namespace shf

// coupled.cu -- the LHMM macro step (coupling protocol Steps 1-4 of
// arXiv 2512.13267): M SPH substeps with the polymer stress held fixed, the
// SPH velocity gradient sent down to every micro-domain, k' DPD steps of
// every box under its gradient, and the time-averaged IK stress sent back up.
// Exchange buffers stay on the device.  The whole macro step can be captured
// once into a CUDA graph (including the micro engine's launches: one
// persistent launch, or size classes on forked streams) and replayed, which removes per-kernel launch overhead from the
// ~60 small SPH launches of each interval.
#include <vector>

#include "lhmm_common.cuh"

// Surrogate gate state (the learned closure is not in the paper).
constexpr int kHist = 16;          // velocity-gradient samples in the closure input
constexpr int kFeat = 4 * kHist + 3;

struct GateState {
  lhmm_closure_t closure = nullptr;
  float threshold = 0.02f;  // relative ensemble spread above which a box runs DPD
  float floor = 1e-3f;      // stress scale floor of the relative spread
  int audit_every = 50;     // every audit_every-th trusted box (round robin) runs DPD anyway
  int absolute = 0;         // 0: closure predicts the increment of pi; 1: pi itself
  int warmup = -1;          // DPD steps a box frozen in the last gated step runs before its
                            // sampled ones when it comes back (-1: the coupling interval k')
  int enabled = 0;
  float* hist = nullptr;    // n x kHist x 4 ring of (Lxx, Lxy, Lyx, Lyy)
  float* X = nullptr;       // n x kFeat closure inputs
  float* mean = nullptr;    // n x 3 predicted increments (xx, xy, yy)
  float* spread = nullptr;  // n
  int* active = nullptr;    // n box list for DPD
  int* n_active = nullptr;  // device count of the list
  long long* counters = nullptr;  // [0] gated steps, [1] DPD boxes, [2] audited boxes, [3] ring head
  double* audit = nullptr;  // [0] sum |pred - dpd|^2, [1] sum |dpd|^2 over audited boxes
  unsigned char* audited = nullptr;  // n
  float* pred = nullptr;    // n x 3 prediction of audited boxes
  float* before = nullptr;  // n x 3 stress before the step of audited boxes
  unsigned char* frozen = nullptr;  // n: box was trusted (not advanced) in the last gated step
  int* resume = nullptr;    // n box list of frozen boxes that run DPD this step
  int* n_resume = nullptr;  // device count of that list
  double* scratch = nullptr;  // n x 6 stress output of the warm-up (discarded)
  // online calibration: trusted boxes take a_k pred_k + c_k per component k,
  // (a, c) the least-squares line of the audited boxes' DPD values on their
  // raw predictions, older macro steps' audits weighted by cal_decay^age
  int online = 0;
  float cal_decay = 0.9f;
  double* cal = nullptr;    // [0..14] decayed sums (n, p, d, pp, pd) x 3; [15..29] this step's
  float* cal_map = nullptr; // (a, c) x 3, read by gate_select
};

struct lhmm_coupled_s {
  lhmm_sph_t sph = nullptr;
  lhmm_micro_t micro = nullptr;
  int sph_substeps = 0, micro_steps = 0, n_boxes = 0;
  float* L_d = nullptr;         // n_boxes x 9, SPH -> micro
  double* stress_d = nullptr;   // n_boxes x 6, micro -> SPH
  cudaStream_t capture_stream = nullptr;
  cudaGraph_t graph[2] = {nullptr, nullptr};      // plain, gated
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  long long steps_done = 0, mode_steps[2] = {0, 0};
  GateState gate;
};

namespace {

// push this step's gradient into the ring and build the closure input
// [L(t-15) .. L(t) as (Lxx, Lxy, Lyx, Lyy), pi_xx, pi_xy, pi_yy]; in the
// absolute mode the stress entries are zero (the input is the history alone)
__global__ void gate_features(const float* L, const double* stress, int n, float* hist,
                              const long long* counters, float* X, int absolute) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= n) return;
  const int head = static_cast<int>(counters[3] % kHist);
  float* h = hist + static_cast<long long>(I) * kHist * 4;
  const float* l = L + 9 * static_cast<long long>(I);
  h[4 * head + 0] = l[0];
  h[4 * head + 1] = l[1];
  h[4 * head + 2] = l[3];
  h[4 * head + 3] = l[4];
  float* x = X + static_cast<long long>(I) * kFeat;
  for (int k = 0; k < kHist; ++k) {
    const int src = (head + 1 + k) % kHist;  // oldest first
    for (int q = 0; q < 4; ++q) x[4 * k + q] = h[4 * src + q];
  }
  const double* s = stress + 6 * static_cast<long long>(I);
  x[4 * kHist + 0] = absolute ? 0.f : static_cast<float>(s[0]);
  x[4 * kHist + 1] = absolute ? 0.f : static_cast<float>(s[3]);
  x[4 * kHist + 2] = absolute ? 0.f : static_cast<float>(s[1]);
}

__global__ void advance_ring(long long* counters) { counters[3] += 1; }

// trust test and compaction; trusted boxes take the prediction (pi += the
// predicted increment, or pi = the predicted stress in the absolute mode),
// the others (and an audit share of the trusted ones) go to the DPD list
__global__ void gate_select(const float* mean, const float* spread, double* stress, int n,
                            float thr, float floor_, int audit_every, int absolute,
                            long long* counters, int* active, int* n_active,
                            unsigned char* audited, float* pred, float* before,
                            unsigned char* frozen, int* resume, int* n_resume,
                            const float* cal_map) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= n) return;
  double* s = stress + 6 * static_cast<long long>(I);
  const float dxx = mean[3 * I], dxy = mean[3 * I + 1], dyy = mean[3 * I + 2];
  // scale: magnitude (Frobenius) of the predicted in-plane stress tensor
  const float bxx = absolute ? 0.f : static_cast<float>(s[0]);
  const float bxy = absolute ? 0.f : static_cast<float>(s[3]);
  const float byy = absolute ? 0.f : static_cast<float>(s[1]);
  const float pxx = bxx + dxx, pxy = bxy + dxy, pyy = byy + dyy;
  const float scale = fmaxf(sqrtf(pxx * pxx + 2.f * pxy * pxy + pyy * pyy), floor_);
  const bool trust = spread[I] <= thr * scale;
  const long long step = counters[0];
  const bool audit = trust && audit_every > 0 && ((I + step) % audit_every) == 0;
  if (!trust || audit) {
    active[atomicAdd(n_active, 1)] = I;
    if (frozen[I]) resume[atomicAdd(n_resume, 1)] = I;  // stale box: warm up first
    frozen[I] = 0;
    if (audit) {
      audited[I] = 1;
      pred[3 * I] = dxx;
      pred[3 * I + 1] = dxy;
      pred[3 * I + 2] = dyy;
      before[3 * I] = bxx;
      before[3 * I + 1] = bxy;
      before[3 * I + 2] = byy;
    }
  } else {
    frozen[I] = 1;
    s[0] = static_cast<double>(bxx) + (cal_map[0] * dxx + cal_map[1]);
    s[3] = static_cast<double>(bxy) + (cal_map[2] * dxy + cal_map[3]);
    s[1] = static_cast<double>(byy) + (cal_map[4] * dyy + cal_map[5]);
  }
}

__global__ void gate_tally(long long* counters, const int* n_active) {
  counters[0] += 1;
  counters[1] += *n_active;
}

__global__ void gate_audit(const double* stress, int n, unsigned char* audited, const float* pred,
                           const float* before, long long* counters, double* audit, double* cal) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= n || !audited[I]) return;
  audited[I] = 0;
  const double* s = stress + 6 * static_cast<long long>(I);
  const double a0 = s[0] - before[3 * I], a1 = s[3] - before[3 * I + 1], a2 = s[1] - before[3 * I + 2];
  const double e0 = pred[3 * I] - a0, e1 = pred[3 * I + 1] - a1, e2 = pred[3 * I + 2] - a2;
  atomicAdd(&audit[0], e0 * e0 + e1 * e1 + e2 * e2);
  atomicAdd(&audit[1], a0 * a0 + a1 * a1 + a2 * a2);
  atomicAdd(reinterpret_cast<unsigned long long*>(&counters[2]), 1ull);
  // this step's sums for the calibration line (raw prediction p, DPD value d)
  const double d[3] = {a0, a1, a2};
  double* step = cal + 15;
  for (int k = 0; k < 3; ++k) {
    const double p = pred[3 * I + k];
    atomicAdd(&step[5 * k + 0], 1.0);
    atomicAdd(&step[5 * k + 1], p);
    atomicAdd(&step[5 * k + 2], d[k]);
    atomicAdd(&step[5 * k + 3], p * p);
    atomicAdd(&step[5 * k + 4], p * d[k]);
  }
}

// fold this step's audit sums into the decayed sums and refit each
// component's line d = a p + c (identity while off, or with fewer than 20
// weighted audits or no spread in p); a is held to [1/4, 4]
__global__ void gate_calibrate(double* cal, float* cal_map, float decay, int online) {
  const int k = threadIdx.x;
  if (k >= 3) return;
  double* run = cal + 5 * k;
  double* step = cal + 15 + 5 * k;
  for (int j = 0; j < 5; ++j) {
    run[j] = static_cast<double>(decay) * run[j] + step[j];
    step[j] = 0.0;
  }
  float a = 1.f, c = 0.f;
  const double w = run[0];
  if (online && w >= 20.0) {
    const double mp = run[1] / w, md = run[2] / w;
    const double vp = run[3] / w - mp * mp, cpd = run[4] / w - mp * md;
    if (vp > 1e-12 * (mp * mp + 1e-30)) {
      const double s = fmin(fmax(cpd / vp, 0.25), 4.0);
      a = static_cast<float>(s);
      c = static_cast<float>(md - s * mp);
    }
  }
  cal_map[2 * k] = a;
  cal_map[2 * k + 1] = c;
}

lhmm_status enqueue_macro_step(lhmm_coupled_s* c, cudaStream_t s, bool gated) {
  lhmm_status st = lhmm_sph_step(c->sph, c->stress_d, c->sph_substeps, c->L_d, s);
  if (st != LHMM_OK) return st;
  GateState& g = c->gate;
  const int n = c->n_boxes, T = 128, G = (n + T - 1) / T;
  if (g.closure) {
    gate_features<<<G, T, 0, s>>>(c->L_d, c->stress_d, n, g.hist, g.counters, g.X, g.absolute);
    advance_ring<<<1, 1, 0, s>>>(g.counters);
    LHMM_CK(cudaGetLastError());
  }
  if (!gated) {
    if (g.closure) LHMM_CK(cudaMemsetAsync(g.frozen, 0, static_cast<size_t>(n), s));  // all advance
    return lhmm_micro_advance(c->micro, c->L_d, nullptr, n, c->micro_steps, c->stress_d, nullptr, s);
  }
  st = lhmm_closure_infer(g.closure, g.X, n, g.mean, g.spread, s);
  if (st != LHMM_OK) return st;
  LHMM_CK(cudaMemsetAsync(g.n_active, 0, sizeof(int), s));
  LHMM_CK(cudaMemsetAsync(g.n_resume, 0, sizeof(int), s));
  gate_select<<<G, T, 0, s>>>(g.mean, g.spread, c->stress_d, n, g.threshold, g.floor, g.audit_every,
                              g.absolute, g.counters, g.active, g.n_active, g.audited, g.pred,
                              g.before, g.frozen, g.resume, g.n_resume, g.cal_map);
  gate_tally<<<1, 1, 0, s>>>(g.counters, g.n_active);
  LHMM_CK(cudaGetLastError());
  const int warm = g.warmup < 0 ? c->micro_steps : g.warmup;
  if (warm > 0) {  // boxes back from a frozen state relax under the current gradient first
    st = lhmm_micro_advance_dev_count(c->micro, c->L_d, g.resume, g.n_resume, n, warm, g.scratch,
                                      nullptr, s);
    if (st != LHMM_OK) return st;
  }
  st = lhmm_micro_advance_dev_count(c->micro, c->L_d, g.active, g.n_active, n, c->micro_steps,
                                    c->stress_d, nullptr, s);
  if (st != LHMM_OK) return st;
  gate_audit<<<G, T, 0, s>>>(c->stress_d, n, g.audited, g.pred, g.before, g.counters, g.audit,
                             g.cal);
  gate_calibrate<<<1, 32, 0, s>>>(g.cal, g.cal_map, g.cal_decay, g.online);
  LHMM_CK(cudaGetLastError());
  return LHMM_OK;
}

void free_gate(GateState& g) {
  cudaFree(g.hist);
  cudaFree(g.X);
  cudaFree(g.mean);
  cudaFree(g.spread);
  cudaFree(g.active);
  cudaFree(g.n_active);
  cudaFree(g.counters);
  cudaFree(g.audit);
  cudaFree(g.audited);
  cudaFree(g.pred);
  cudaFree(g.before);
  cudaFree(g.frozen);
  cudaFree(g.resume);
  cudaFree(g.n_resume);
  cudaFree(g.scratch);
  cudaFree(g.cal);
  cudaFree(g.cal_map);
  g = GateState();
}

void drop_graphs(lhmm_coupled_s* c) {
  for (int m = 0; m < 2; ++m) {
    if (c->exec[m]) cudaGraphExecDestroy(c->exec[m]);
    if (c->graph[m]) cudaGraphDestroy(c->graph[m]);
    c->exec[m] = nullptr;
    c->graph[m] = nullptr;
    c->mode_steps[m] = 0;
  }
}

void free_coupled(lhmm_coupled_s* c) {
  if (!c) return;
  drop_graphs(c);
  if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
  cudaFree(c->L_d);
  cudaFree(c->stress_d);
  free_gate(c->gate);
  delete c;
}

}  // namespace

extern "C" lhmm_status lhmm_coupled_create(lhmm_sph_t sph, lhmm_micro_t micro, int sph_substeps,
                                           int micro_steps, lhmm_coupled_t* out) {
  if (!sph || !micro || !out || sph_substeps < 1 || micro_steps < 1) return LHMM_ERR_ARG;
  *out = nullptr;
  int n = 0, n_wall = 0, nb = 0;
  int64_t beads = 0;
  int mx = 0;
  lhmm_status st = lhmm_sph_info(sph, &n, &n_wall);
  if (st != LHMM_OK) return st;
  st = lhmm_micro_info(micro, &nb, &beads, &mx);
  if (st != LHMM_OK) return st;
  if (nb != n - n_wall) return LHMM_ERR_ARG;  // one box per fluid particle
  lhmm_coupled_s* c = new lhmm_coupled_s();
  c->sph = sph;
  c->micro = micro;
  c->sph_substeps = sph_substeps;
  c->micro_steps = micro_steps;
  c->n_boxes = nb;
  cudaError_t e;
  const size_t nbx = static_cast<size_t>(nb > 0 ? nb : 1);
  if ((e = cudaMalloc(&c->L_d, sizeof(float) * 9 * nbx)) != cudaSuccess ||
      (e = cudaMalloc(&c->stress_d, sizeof(double) * 6 * nbx)) != cudaSuccess ||
      (e = cudaMemset(c->L_d, 0, sizeof(float) * 9 * nbx)) != cudaSuccess ||
      (e = cudaMemset(c->stress_d, 0, sizeof(double) * 6 * nbx)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking)) != cudaSuccess) {
    free_coupled(c);
    return lhmm_cuda_error(e);
  }
  *out = c;
  return LHMM_OK;
}

extern "C" lhmm_status lhmm_coupled_destroy(lhmm_coupled_t c) {
  if (!c) return LHMM_ERR_ARG;
  cudaDeviceSynchronize();
  free_coupled(c);
  return LHMM_OK;
}

extern "C" lhmm_status lhmm_coupled_step(lhmm_coupled_t c, int n_macro, int use_graph,
                                         void* stream) {
  if (!c || n_macro < 0) return LHMM_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool gated = c->gate.closure && c->gate.enabled;
  const int mode = gated ? 1 : 0;
  for (int k = 0; k < n_macro; ++k) {
    if (!use_graph || c->mode_steps[mode] == 0) {
      // eager (the first step of a mode also sets kernel attributes and grows
      // workspaces before any capture)
      lhmm_status st = enqueue_macro_step(c, s, gated);
      if (st != LHMM_OK) return st;
    } else {
      if (!c->exec[mode]) {
        LHMM_CK(cudaStreamSynchronize(s));
        LHMM_CK(cudaStreamBeginCapture(c->capture_stream, cudaStreamCaptureModeThreadLocal));
        lhmm_status st = enqueue_macro_step(c, c->capture_stream, gated);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(c->capture_stream, &g);
        if (st != LHMM_OK) {
          if (g) cudaGraphDestroy(g);
          return st;
        }
        if (e != cudaSuccess) return lhmm_cuda_error(e);
        c->graph[mode] = g;
        e = cudaGraphInstantiate(&c->exec[mode], g, 0);
        if (e != cudaSuccess) {
          c->exec[mode] = nullptr;
          return lhmm_cuda_error(e);
        }
      }
      LHMM_CK(cudaGraphLaunch(c->exec[mode], s));
    }
    ++c->mode_steps[mode];
    ++c->steps_done;
  }
  return LHMM_OK;
}

extern "C" lhmm_status lhmm_coupled_set_closure(lhmm_coupled_t c, lhmm_closure_t closure,
                                                float threshold, float stress_floor,
                                                int audit_every) {
  if (!c || !closure || !(threshold >= 0.f) || !(stress_floor > 0.f) || audit_every < 0)
    return LHMM_ERR_ARG;
  LHMM_CK(cudaDeviceSynchronize());
  drop_graphs(c);
  free_gate(c->gate);
  GateState& g = c->gate;
  const size_t n = static_cast<size_t>(c->n_boxes > 0 ? c->n_boxes : 1);
  cudaError_t e;
  if ((e = cudaMalloc(&g.hist, sizeof(float) * n * kHist * 4)) != cudaSuccess ||
      (e = cudaMalloc(&g.X, sizeof(float) * n * kFeat)) != cudaSuccess ||
      (e = cudaMalloc(&g.mean, sizeof(float) * n * 3)) != cudaSuccess ||
      (e = cudaMalloc(&g.spread, sizeof(float) * n)) != cudaSuccess ||
      (e = cudaMalloc(&g.active, sizeof(int) * n)) != cudaSuccess ||
      (e = cudaMalloc(&g.n_active, sizeof(int))) != cudaSuccess ||
      (e = cudaMalloc(&g.counters, sizeof(long long) * 4)) != cudaSuccess ||
      (e = cudaMalloc(&g.audit, sizeof(double) * 2)) != cudaSuccess ||
      (e = cudaMalloc(&g.audited, n)) != cudaSuccess ||
      (e = cudaMalloc(&g.pred, sizeof(float) * n * 3)) != cudaSuccess ||
      (e = cudaMalloc(&g.before, sizeof(float) * n * 3)) != cudaSuccess ||
      (e = cudaMalloc(&g.frozen, n)) != cudaSuccess ||
      (e = cudaMalloc(&g.resume, sizeof(int) * n)) != cudaSuccess ||
      (e = cudaMalloc(&g.n_resume, sizeof(int))) != cudaSuccess ||
      (e = cudaMalloc(&g.scratch, sizeof(double) * n * 6)) != cudaSuccess ||
      (e = cudaMalloc(&g.cal, sizeof(double) * 30)) != cudaSuccess ||
      (e = cudaMalloc(&g.cal_map, sizeof(float) * 6)) != cudaSuccess ||
      (e = cudaMemset(g.cal, 0, sizeof(double) * 30)) != cudaSuccess ||
      (e = cudaMemset(g.frozen, 0, n)) != cudaSuccess ||
      (e = cudaMemset(g.hist, 0, sizeof(float) * n * kHist * 4)) != cudaSuccess ||
      (e = cudaMemset(g.counters, 0, sizeof(long long) * 4)) != cudaSuccess ||
      (e = cudaMemset(g.audit, 0, sizeof(double) * 2)) != cudaSuccess ||
      (e = cudaMemset(g.audited, 0, n)) != cudaSuccess ||
      (e = cudaMemset(g.n_active, 0, sizeof(int))) != cudaSuccess) {
    free_gate(g);
    return lhmm_cuda_error(e);
  }
  const float identity[6] = {1.f, 0.f, 1.f, 0.f, 1.f, 0.f};
  if ((e = cudaMemcpy(g.cal_map, identity, sizeof(identity), cudaMemcpyHostToDevice)) != cudaSuccess) {
    free_gate(g);
    return lhmm_cuda_error(e);
  }
  g.closure = closure;
  g.threshold = threshold;
  g.floor = stress_floor;
  g.audit_every = audit_every;
  g.enabled = 0;
  return LHMM_OK;
}

extern "C" lhmm_status lhmm_coupled_set_gate(lhmm_coupled_t c, float threshold, int audit_every,
                                             int absolute, int warmup_steps) {
  if (!c || !c->gate.closure || !(threshold >= 0.f) || audit_every < 0 ||
      (absolute != 0 && absolute != 1) || warmup_steps < -1)
    return LHMM_ERR_ARG;
  LHMM_CK(cudaDeviceSynchronize());
  drop_graphs(c);  // the gate's launch arguments are baked into the captured graph
  c->gate.threshold = threshold;
  c->gate.audit_every = audit_every;
  c->gate.absolute = absolute;
  c->gate.warmup = warmup_steps;
  return LHMM_OK;
}

extern "C" lhmm_status lhmm_coupled_set_online_calibration(lhmm_coupled_t c, int enabled,
                                                          float decay, float* map_host) {
  if (!c || !c->gate.closure || (enabled != 0 && enabled != 1 && enabled != -1) ||
      !(decay > 0.f && decay <= 1.f))
    return LHMM_ERR_ARG;
  LHMM_CK(cudaDeviceSynchronize());
  if (map_host) LHMM_CK(cudaMemcpy(map_host, c->gate.cal_map, sizeof(float) * 6, cudaMemcpyDeviceToHost));
  if (enabled == -1) return LHMM_OK;  // read only
  drop_graphs(c);  // the flag and the decay are launch arguments of a captured graph
  c->gate.online = enabled;
  c->gate.cal_decay = decay;
  return LHMM_OK;
}

extern "C" lhmm_status lhmm_coupled_enable_gate(lhmm_coupled_t c, int enabled) {
  if (!c || !c->gate.closure) return LHMM_ERR_ARG;
  c->gate.enabled = enabled ? 1 : 0;
  return LHMM_OK;
}

extern "C" lhmm_status lhmm_coupled_gate_stats(lhmm_coupled_t c, int64_t* gated_steps,
                                               int64_t* dpd_boxes, int64_t* audited_boxes,
                                               double* audit_err2, double* audit_ref2) {
  if (!c || !c->gate.closure) return LHMM_ERR_ARG;
  LHMM_CK(cudaDeviceSynchronize());
  long long cnt[4];
  double au[2];
  LHMM_CK(cudaMemcpy(cnt, c->gate.counters, sizeof(cnt), cudaMemcpyDeviceToHost));
  LHMM_CK(cudaMemcpy(au, c->gate.audit, sizeof(au), cudaMemcpyDeviceToHost));
  if (gated_steps) *gated_steps = cnt[0];
  if (dpd_boxes) *dpd_boxes = cnt[1];
  if (audited_boxes) *audited_boxes = cnt[2];
  if (audit_err2) *audit_err2 = au[0];
  if (audit_ref2) *audit_ref2 = au[1];
  return LHMM_OK;
}

extern "C" lhmm_status lhmm_coupled_closure_inputs(lhmm_coupled_t c, float* X_host) {
  if (!c || !c->gate.closure || !X_host) return LHMM_ERR_ARG;
  LHMM_CK(cudaDeviceSynchronize());
  LHMM_CK(cudaMemcpy(X_host, c->gate.X, sizeof(float) * c->n_boxes * kFeat, cudaMemcpyDeviceToHost));
  return LHMM_OK;
}

extern "C" lhmm_status lhmm_coupled_exchange(lhmm_coupled_t c, float** L_dev, double** stress_dev) {
  if (!c) return LHMM_ERR_ARG;
  if (L_dev) *L_dev = c->L_d;
  if (stress_dev) *stress_dev = c->stress_d;
  return LHMM_OK;
}

extern "C" lhmm_status lhmm_coupled_copy_exchange(lhmm_coupled_t c, float* L_host,
                                                  double* stress_host) {
  if (!c) return LHMM_ERR_ARG;
  LHMM_CK(cudaDeviceSynchronize());
  const size_t nb = static_cast<size_t>(c->n_boxes);
  if (L_host) LHMM_CK(cudaMemcpy(L_host, c->L_d, sizeof(float) * 9 * nb, cudaMemcpyDeviceToHost));
  if (stress_host)
    LHMM_CK(cudaMemcpy(stress_host, c->stress_d, sizeof(double) * 6 * nb, cudaMemcpyDeviceToHost));
  return LHMM_OK;
}

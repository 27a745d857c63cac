// coupled.cu -- the LHMM macro step (coupling protocol Steps 1-4 of
// arXiv 2512.13267): M SPH substeps with the polymer stress held fixed, the
// SPH velocity gradient sent down to every micro-domain, k' DPD steps of
// every box under its gradient, and the time-averaged IK stress sent back up.
// Exchange buffers stay on the device.  The whole macro step can be captured
// once into a CUDA graph (including the micro engine's forked size-class
// streams) and replayed, which removes per-kernel launch overhead from the
// ~60 small SPH launches of each interval.
#include <vector>

#include "lhmm_common.cuh"

struct lhmm_coupled_s {
  lhmm_sph_t sph = nullptr;
  lhmm_micro_t micro = nullptr;
  int sph_substeps = 0, micro_steps = 0, n_boxes = 0;
  float* L_d = nullptr;         // n_boxes x 9, SPH -> micro
  double* stress_d = nullptr;   // n_boxes x 6, micro -> SPH
  cudaStream_t capture_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  long long steps_done = 0;
};

namespace {

lhmm_status enqueue_macro_step(lhmm_coupled_s* c, cudaStream_t s) {
  lhmm_status st = lhmm_sph_step(c->sph, c->stress_d, c->sph_substeps, c->L_d, s);
  if (st != LHMM_OK) return st;
  return lhmm_micro_advance(c->micro, c->L_d, nullptr, c->n_boxes, c->micro_steps, c->stress_d,
                            nullptr, s);
}

void free_coupled(lhmm_coupled_s* c) {
  if (!c) return;
  if (c->exec) cudaGraphExecDestroy(c->exec);
  if (c->graph) cudaGraphDestroy(c->graph);
  if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
  cudaFree(c->L_d);
  cudaFree(c->stress_d);
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
  for (int k = 0; k < n_macro; ++k) {
    if (!use_graph || c->steps_done == 0) {
      // eager (the first step also sets kernel attributes before any capture)
      lhmm_status st = enqueue_macro_step(c, s);
      if (st != LHMM_OK) return st;
    } else {
      if (!c->exec) {
        LHMM_CK(cudaStreamSynchronize(s));
        LHMM_CK(cudaStreamBeginCapture(c->capture_stream, cudaStreamCaptureModeThreadLocal));
        lhmm_status st = enqueue_macro_step(c, c->capture_stream);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(c->capture_stream, &g);
        if (st != LHMM_OK) {
          if (g) cudaGraphDestroy(g);
          return st;
        }
        if (e != cudaSuccess) return lhmm_cuda_error(e);
        c->graph = g;
        e = cudaGraphInstantiate(&c->exec, g, 0);
        if (e != cudaSuccess) {
          c->exec = nullptr;
          return lhmm_cuda_error(e);
        }
      }
      LHMM_CK(cudaGraphLaunch(c->exec, s));
    }
    ++c->steps_done;
  }
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

// api.cu -- status strings and CUDA error mapping of the LHMM C ABI.
#include "lhmm_common.cuh"

lhmm_status lhmm_cuda_error(cudaError_t e) {
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return LHMM_ERR_OOM;
  }
  return LHMM_ERR_CUDA;
}

extern "C" const char* lhmm_status_string(lhmm_status s) {
  switch (s) {
    case LHMM_OK: return "ok";
    case LHMM_ERR_ARG: return "invalid argument";
    case LHMM_ERR_CUDA: return "CUDA runtime error";
    case LHMM_ERR_OOM: return "device out of memory";
    case LHMM_ERR_BOND_OVERSTRETCH: return "FENE bond reached R0";
    case LHMM_ERR_CELL_OVERFLOW: return "box exceeded its cell/shared-memory plan";
    case LHMM_ERR_NAN: return "non-finite bead state";
    case LHMM_ERR_TIMEOUT: return "bounded device wait timed out";
    case LHMM_ERR_UNSUPPORTED: return "unsupported configuration";
    case LHMM_ERR_FORCE_RANGE: return "pair force out of fixed-point range (clamped)";
  }
  return "unknown status";
}

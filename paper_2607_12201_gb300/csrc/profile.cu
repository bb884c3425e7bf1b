// Measurement hooks: CUDA-event timing of individual phases of the hot path
// on the problem's stream, and a fused-multiply-add throughput probe that
// gives the arithmetic roof for the FP64 / FP32 element factorization.
#include <algorithm>

#include "problem.cuh"

namespace collo {

// Each thread runs 8 independent FMA chains of `iters` steps; the result is
// stored so the work cannot be removed.
template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(T* __restrict__ out, int iters, T a, T b) {
  T v[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = (T)(threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = v[k] * a + b;
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += v[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace collo

using namespace collo;

extern "C" {

collo_status collo_alu_peak(int precision, double* tflops) {
  if (!tflops) { set_error("NULL argument"); return COLLO_ERR_INVALID_ARG; }
  int dev = 0, sms = 0;
  COLLO_CUDA(cudaGetDevice(&dev));
  COLLO_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8, threads = 256;
  const int iters = precision == COLLO_PRECISION_FP64 ? 4096 : 65536;
  void* buf = nullptr;
  COLLO_CUDA(cudaMalloc(&buf, (size_t)blocks * threads * sizeof(double)));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(e0);
    count_launch();
    if (precision == COLLO_PRECISION_FP64)
      k_fma_probe<double><<<blocks, threads>>>((double*)buf, iters, 0.999999, 1e-7);
    else
      k_fma_probe<float><<<blocks, threads>>>((float*)buf, iters, 0.999999f, 1e-7f);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0) best = std::min(best, ms);
  }
  cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  if (err != cudaSuccess) { set_error(cudaGetErrorString(err)); return COLLO_ERR_DEVICE; }
  const double flops = 2.0 * 8.0 * (double)iters * blocks * threads;
  *tflops = flops / (best * 1e-3) / 1e12;
  return COLLO_OK;
}

collo_status collo_time_phase(collo_problem* prob, int phase, int precision, int reps,
                              double* ms_per_launch) {
  if (!prob || !ms_per_launch || reps < 1) { set_error("bad argument"); return COLLO_ERR_INVALID_ARG; }
  if (!prob->evaluated) { set_error("collo_eval has not run"); return COLLO_ERR_NOT_EVALUATED; }
  COLLO_CUDA(cudaSetDevice(prob->device));
  if (phase >= 5 && phase <= 7) {   // lifted path
    collo_status s = lifted_time_launch(prob, phase - 5);   // warm-up, checks the state
    if (s != COLLO_OK) return s;
    cudaEvent_t e0, e1;
    COLLO_CUDA(cudaEventCreate(&e0));
    COLLO_CUDA(cudaEventCreate(&e1));
    COLLO_CUDA(cudaEventRecord(e0, prob->stream));
    for (int k = 0; k < reps && s == COLLO_OK; ++k) s = lifted_time_launch(prob, phase - 5);
    COLLO_CUDA(cudaEventRecord(e1, prob->stream));
    COLLO_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms_per_launch = ms / reps;
    return s;
  }
  if (precision < 0) precision = prob->precision;
  collo_status s = ensure_factor_storage(prob, precision);
  if (s != COLLO_OK) return s;
  cudaStream_t st = prob->stream;
  const bool mixed = precision == COLLO_PRECISION_MIXED;
  if ((phase == 2) && prob->factored != precision) {
    set_error("phase 2 (solve) needs a factorization in this precision");
    return COLLO_ERR_NOT_FACTORED;
  }
  if (phase >= 1 && phase <= 3) return runner_time_phase(prob, phase, precision, reps, ms_per_launch);
  auto launch = [&]() -> cudaError_t {
    switch (phase) {
      case 0:
        return mixed ? launch_elem_factor<float>(prob->P, prob->E, prob->sigma, prob->fac_dw,
                                                 prob->fac_dc, prob->f32.F, st)
                     : launch_elem_factor<double>(prob->P, prob->E, prob->sigma, prob->fac_dw,
                                                  prob->fac_dc, prob->f64.F, st);
      case 4:
        return launch_forward_sweep(prob);
      default:
        return cudaErrorInvalidValue;
    }
  };
  COLLO_CUDA(launch());   // warm-up
  cudaEvent_t e0, e1;
  COLLO_CUDA(cudaEventCreate(&e0));
  COLLO_CUDA(cudaEventCreate(&e1));
  COLLO_CUDA(cudaEventRecord(e0, st));
  for (int k = 0; k < reps; ++k) COLLO_CUDA(launch());
  COLLO_CUDA(cudaEventRecord(e1, st));
  COLLO_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms_per_launch = ms / reps;
  // the factorization storage now holds the re-run phase; keep it consistent
  if (phase == 0) prob->factored = -1;
  return COLLO_OK;
}

}  // extern "C"

// Throughput of the float64 operations the edge cost (Eq. 1) is made of, on
// the current device: fused multiply-adds, divisions and square roots.  The
// cost kernel is bound by the float64 pipe, and on this GPU a float64
// division or square root is a sequence of pipe instructions rather than
// one, so the roofline of that kernel needs these rates measured, not only
// the FMA peak.  Measurement support; nothing of the simplification uses it.
//
// Each kernel runs one full wave of independent chains.  Division and square
// root are timed against a loop with the same float64 additions and no
// division or root, and the difference is charged to the operation.
#include "common.cuh"

namespace pamo {

namespace {

constexpr int kProbeBlock = 256;

__global__ void __launch_bounds__(kProbeBlock) k_probe_fma(double* __restrict__ out, int iters,
                                                           double a, double b) {
  double x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  double x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; i++) {
    x0 = __fma_rn(x0, a, b); x1 = __fma_rn(x1, a, b); x2 = __fma_rn(x2, a, b);
    x3 = __fma_rn(x3, a, b); x4 = __fma_rn(x4, a, b); x5 = __fma_rn(x5, a, b);
    x6 = __fma_rn(x6, a, b); x7 = __fma_rn(x7, a, b);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

// op: 0 = the additions alone, 1 = with a division, 2 = with a square root
__global__ void __launch_bounds__(kProbeBlock) k_probe_op(double* __restrict__ out, int iters,
                                                          int op, double a) {
  double x = threadIdx.x + 1.0;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  for (int i = 0; i < iters; i++) {
    const double y0 = x, y1 = x + 0.25, y2 = x + 0.5, y3 = x + 0.75;
    if (op == 1) {
      s0 += a / y0; s1 += a / y1; s2 += a / y2; s3 += a / y3;
    } else if (op == 2) {
      s0 += sqrt(y0); s1 += sqrt(y1); s2 += sqrt(y2); s3 += sqrt(y3);
    } else {
      s0 += y0; s1 += y1; s2 += y2; s3 += y3;
    }
    x += 1.0;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = s0 + s1 + s2 + s3;
}

}  // namespace

}  // namespace pamo

using namespace pamo;

extern "C" pamo_status pamo_measure_fp64(void* stream, double* h_rates) {
  if (!h_rates) {
    set_error("pamo_measure_fp64: h_rates required");
    return PAMO_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int per_sm = 0;
  PAMO_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_probe_op, kProbeBlock, 0));
  const int blocks = sm_count() * (per_sm > 0 ? per_sm : 1);
  const int64_t threads = (int64_t)blocks * kProbeBlock;
  double* out = nullptr;
  PAMO_CUDA(cudaMallocAsync((void**)&out, sizeof(double) * (size_t)threads, st));
  cudaEvent_t e0, e1;
  PAMO_CUDA(cudaEventCreate(&e0));
  PAMO_CUDA(cudaEventCreate(&e1));
  constexpr int kFmaIters = 4096, kOpIters = 1024;
  float ms[4] = {0.f, 0.f, 0.f, 0.f};
  pamo_status s = PAMO_OK;
  for (int rep = 0; rep < 2 && s == PAMO_OK; rep++) {  // the first pass warms up
    for (int k = 0; k < 4 && s == PAMO_OK; k++) {
      cudaError_t e = cudaEventRecord(e0, st);
      if (k == 0) k_probe_fma<<<blocks, kProbeBlock, 0, st>>>(out, kFmaIters, 0.999, 1e-3);
      else k_probe_op<<<blocks, kProbeBlock, 0, st>>>(out, kOpIters, k - 1, 3.0);
      note_launch();
      if (e == cudaSuccess) e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaEventRecord(e1, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms[k], e0, e1);
      if (e != cudaSuccess) s = cuda_fail(e, "float64 probe");
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(out, st);
  cudaStreamSynchronize(st);
  if (s != PAMO_OK) return s;
  const double n_fma = 8.0 * kFmaIters * (double)threads;
  const double n_op = 4.0 * kOpIters * (double)threads;
  h_rates[0] = n_fma / (ms[0] * 1e-3);
  // time beyond the same loop of additions; a difference at or below zero
  // (not expected) reports 0
  const double t_div = (ms[2] - ms[1]) * 1e-3, t_sqrt = (ms[3] - ms[1]) * 1e-3;
  h_rates[1] = t_div > 0.0 ? n_op / t_div : 0.0;
  h_rates[2] = t_sqrt > 0.0 ? n_op / t_sqrt : 0.0;
  return PAMO_OK;
}

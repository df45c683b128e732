// Measurement utility: the L2 read bandwidth of the current GPU, the
// denominator of the on-chip roofline of kernels whose working set (a BVH, an
// environment map) stays in L2.  Not part of the method.
#include <cuda_runtime.h>
#include <stdint.h>

#include "dt_internal.cuh"

namespace dt {

// Every thread streams float4 loads that bypass L1 (ld.global.cg) over a
// buffer small enough to stay in L2, `iters` times.
__global__ void k_l2_read(const float4* __restrict__ p, size_t n4, int iters, float* __restrict__ sink) {
  float acc = 0.f;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (int it = 0; it < iters; ++it) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += stride) {
      const float4 v = __ldcg(p + i);
      acc += v.x + v.y + v.z + v.w;
    }
  }
  if (acc == 1234.5f) sink[0] = acc;  // keeps the loads alive
}

}  // namespace dt

using namespace dt;

extern "C" dt_status dt_measure_l2_read_bandwidth(const void* d_buf, size_t bytes, int32_t iters, double* gbps,
                                                  dt_stream stream) {
  if (!d_buf || !gbps || bytes < 4096 || iters < 1) return set_error(DT_ERR_INVALID_ARG, "bad argument");
  if (((uintptr_t)d_buf % 16) != 0) return set_error(DT_ERR_INVALID_ARG, "buffer must be 16-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n4 = bytes / 16;
  float* sink = (float*)d_buf;  // never written in practice (see k_l2_read)
  const int blocks = 4 * num_sms();
  k_l2_read<<<blocks, 512, 0, s>>>((const float4*)d_buf, n4, 1, sink);  // warm the lines into L2
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e == cudaSuccess) e = cudaEventRecord(a, s);
  if (e == cudaSuccess) k_l2_read<<<blocks, 512, 0, s>>>((const float4*)d_buf, n4, iters, sink);
  if (e == cudaSuccess) e = cudaEventRecord(b, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (e != cudaSuccess) return set_error(DT_ERR_CUDA, "dt_measure_l2_read_bandwidth: %s", cudaGetErrorString(e));
  *gbps = (double)n4 * 16.0 * iters / (ms * 1e-3) / 1e9;
  return check_launch("dt_measure_l2_read_bandwidth");
}

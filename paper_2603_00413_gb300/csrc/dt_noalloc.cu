// dt_vertex_normals_noalloc: the vertex normals of dt_vertex_normals for
// callers that cannot allocate device memory themselves.
//
// Who needs it: a caller that only receives device pointers from a host
// application that owns all device memory (a plugin with no allocation hook),
// or a serving loop that must not allocate after start-up (cudaMalloc and
// cudaFree can synchronise the device and fragment a memory pool), cannot
// hand dt_vertex_normals the scratch buffer it needs.  This entry point keeps
// that scratch in a fixed array of device memory inside the library, so the
// caller passes only its inputs and outputs.
//
// The array is a file-scope static __device__ variable of kNoAllocMaxVertices
// * 3 64-bit words (24 MiB).  Every GPU that loads the library holds it until
// the process exits.  Host code cannot use the array's name as a device
// address, so the first call on each device looks the address up with
// cudaGetSymbolAddress (with that device current) and keeps it.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "dt_internal.cuh"

namespace dt {

// the kernels of dt_vertex_normals (dt_bvh.cu), given this file's scratch
__global__ void k_face_normals_scatter(const float* __restrict__ V, const int32_t* __restrict__ F, int32_t nf,
                                       unsigned long long* __restrict__ acc);
__global__ void k_normals_finish(const unsigned long long* __restrict__ acc, int64_t n3, float* __restrict__ N);

constexpr int32_t kNoAllocMaxVertices = 1 << 20;

// fixed-point accumulators of the normal sums, 3 per vertex
static __device__ __align__(256) unsigned long long g_normals_scratch[(size_t)kNoAllocMaxVertices * 3];

namespace {
std::mutex g_noalloc_mu;
unsigned long long* g_noalloc_ptr[64] = {nullptr};

// Device address of the array on the current device (looked up once per
// device).
dt_status noalloc_scratch(unsigned long long** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(DT_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= 64) return set_error(DT_ERR_INVALID_ARG, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_normals_scratch);
    if (e != cudaSuccess || !p)
      return set_error(DT_ERR_CUDA, "cudaGetSymbolAddress of the normals scratch: %s", cudaGetErrorString(e));
    g_noalloc_ptr[dev] = (unsigned long long*)p;
  }
  *out = g_noalloc_ptr[dev];
  return DT_OK;
}
}  // namespace

}  // namespace dt

using namespace dt;

extern "C" dt_status dt_vertex_normals_noalloc(const float* d_V, int32_t nv, const int32_t* d_F, int32_t nf,
                                               float* d_N, dt_stream stream) {
  if (!d_V || !d_F || !d_N) return set_error(DT_ERR_INVALID_ARG, "NULL pointer");
  if (nv < 1 || nf < 1) return set_error(DT_ERR_INVALID_ARG, "nv and nf must be >= 1");
  if (nv > kNoAllocMaxVertices)
    return set_error(DT_ERR_INVALID_ARG,
                     "dt_vertex_normals_noalloc handles at most %d vertices (got %d); use dt_vertex_normals "
                     "with a caller scratch buffer", kNoAllocMaxVertices, nv);
  unsigned long long* acc = nullptr;
  dt_status st = noalloc_scratch(&acc);
  if (st != DT_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  // the array keeps the previous call's sums: clear the part this call uses
  cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * 3 * (size_t)nv, s);
  if (e != cudaSuccess) return set_error(DT_ERR_CUDA, "clearing the normals scratch: %s", cudaGetErrorString(e));
  const int cap = 4 * num_sms();
  const int b1 = (int)((nf + 255) / 256) < cap ? (int)((nf + 255) / 256) : cap;
  k_face_normals_scatter<<<b1 > 0 ? b1 : 1, 256, 0, s>>>(d_V, d_F, nf, acc);
  const int64_t n3 = 3 * (int64_t)nv;
  const int b2 = (int)((n3 + 255) / 256) < cap ? (int)((n3 + 255) / 256) : cap;
  k_normals_finish<<<b2 > 0 ? b2 : 1, 256, 0, s>>>(acc, n3, d_N);
  return check_launch("dt_vertex_normals_noalloc");
}

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
// address, so the first call in each CUDA context (one per device, unless
// the context is destroyed and made again, as cudaDeviceReset does) looks the
// address up with cudaGetSymbolAddress, with that device current, and keeps
// it for that context.
#include <cuda.h>
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
// The array's address is a property of the module loaded into one CUDA
// context: a context made anew (cudaDeviceReset, then any call) loads the
// module again, possibly elsewhere.  So the cache is keyed on the context's
// id, which the driver never gives to another context in this process.  The
// two driver calls are reached through the runtime's entry-point query, so
// the library does not link the driver library itself.
typedef CUresult (*PfnCtxGetCurrent)(CUcontext*);
typedef CUresult (*PfnCtxGetId)(CUcontext, unsigned long long*);

constexpr int kCacheSlots = 64;
struct CacheSlot {
  unsigned long long ctx_id;
  unsigned long long* ptr;
};

std::mutex g_noalloc_mu;
CacheSlot g_noalloc_cache[kCacheSlots] = {};
int g_noalloc_used = 0;
PfnCtxGetCurrent g_ctx_get_current = nullptr;
PfnCtxGetId g_ctx_get_id = nullptr;

dt_status resolve_driver_calls() {
  if (g_ctx_get_current && g_ctx_get_id) return DT_OK;
  void* f1 = nullptr;
  void* f2 = nullptr;
  cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = cudaDriverEntryPointSymbolNotFound;
  cudaError_t e1 = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
  cudaError_t e2 = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
  if (e1 != cudaSuccess || e2 != cudaSuccess || q1 != cudaDriverEntryPointSuccess ||
      q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
    return set_error(DT_ERR_CUDA, "looking up cuCtxGetCurrent/cuCtxGetId: %s",
                     cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
  g_ctx_get_current = (PfnCtxGetCurrent)f1;
  g_ctx_get_id = (PfnCtxGetId)f2;
  return DT_OK;
}

// Id of the current context; *id = 0 when no context is current yet.
dt_status current_context_id(unsigned long long* id) {
  CUcontext ctx = nullptr;
  CUresult r = g_ctx_get_current(&ctx);
  if (r != CUDA_SUCCESS) return set_error(DT_ERR_CUDA, "cuCtxGetCurrent failed (%d)", (int)r);
  *id = 0;
  if (!ctx) return DT_OK;
  r = g_ctx_get_id(ctx, id);
  if (r != CUDA_SUCCESS) return set_error(DT_ERR_CUDA, "cuCtxGetId failed (%d)", (int)r);
  return DT_OK;
}

// Device address of the array in the current context (looked up once per
// context, with the context's device current).
dt_status noalloc_scratch(unsigned long long** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(DT_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  dt_status st = resolve_driver_calls();
  if (st != DT_OK) return st;
  unsigned long long id = 0;
  st = current_context_id(&id);
  if (st != DT_OK) return st;
  if (id) {
    for (int i = 0; i < g_noalloc_used; ++i)
      if (g_noalloc_cache[i].ctx_id == id) {
        *out = g_noalloc_cache[i].ptr;
        return DT_OK;
      }
  }
  // set-up for this context: the symbol lookup also makes the device's
  // primary context current if no context was yet
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_normals_scratch);
  if (e != cudaSuccess || !p)
    return set_error(DT_ERR_CUDA, "cudaGetSymbolAddress of the normals scratch: %s", cudaGetErrorString(e));
  if (!id) {
    st = current_context_id(&id);
    if (st != DT_OK) return st;
  }
  if (id) {
    if (g_noalloc_used < kCacheSlots) {
      g_noalloc_cache[g_noalloc_used++] = CacheSlot{id, (unsigned long long*)p};
    } else {  // more contexts than slots in one process: reuse the oldest slot
      for (int i = 1; i < kCacheSlots; ++i) g_noalloc_cache[i - 1] = g_noalloc_cache[i];
      g_noalloc_cache[kCacheSlots - 1] = CacheSlot{id, (unsigned long long*)p};
    }
  }
  *out = (unsigned long long*)p;
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

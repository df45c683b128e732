// Geometry kernels: vertex normals (DiffTrans Sec. 3.4, Eq. 13) and their
// backward, and the LBVH (Morton codes, a stable LSD radix sort, the Karras
// 2012 hierarchy, bottom-up bounds written straight into the float4 node
// layout that the traversal reads).
#include <cuda_runtime.h>
#include <stdint.h>

#include "dt_internal.cuh"
#include "dt_shade.cuh"

namespace dt {

extern dt_tuning g_tuning;

// ---------------------------------------------------------------------------
// Eq. 13: N_v = (1/3) sum_{f containing v} unit((v1 - v0) x (v2 - v0)).
// One thread per face adds its unit normal, in 2^-40 fixed point, to its
// three vertices with 64-bit integer atomics: integer addition is
// associative, so the sums -- and every ray that depends on them -- are the
// same bits on every run whatever order the atomics land in.  A second pass
// converts to float and applies the 1/3.  Both conversions are FP32: the
// scale is a power of two, so u * 2^40 is exact in float (|u| <= 1) and the
// integer is u's value rounded to 2^-40; the finish rounds the sum to float
// once and divides by 3 with IEEE rounding.
// ---------------------------------------------------------------------------
constexpr float kNormalFix = 0x1p40f;
constexpr float kNormalUnfix = 0x1p-40f;

__global__ void k_face_normals_scatter(const float* __restrict__ V, const int32_t* __restrict__ F, int32_t nf,
                                       unsigned long long* __restrict__ acc) {
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += gridDim.x * blockDim.x) {
    const int i0 = F[3 * f], i1 = F[3 * f + 1], i2 = F[3 * f + 2];
    const float3 v0 = load3(V + 3 * i0), v1 = load3(V + 3 * i1), v2 = load3(V + 3 * i2);
    const float3 c = cross_rn(v1 - v0, v2 - v0);
    const float lc = len(c);
    if (!(lc > 0.0f)) continue;  // a zero-area face has no unit normal and adds nothing
    const float3 u = mk(c.x / lc, c.y / lc, c.z / lc);
    const long long q[3] = {__float2ll_rn(u.x * kNormalFix), __float2ll_rn(u.y * kNormalFix),
                            __float2ll_rn(u.z * kNormalFix)};
    const int idx[3] = {i0, i1, i2};
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int c = 0; c < 3; ++c) atomicAdd(acc + 3 * (size_t)idx[k] + c, (unsigned long long)q[c]);
  }
}

__global__ void k_normals_finish(const unsigned long long* __restrict__ acc, int64_t n3, float* __restrict__ N) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x)
    N[i] = __fdiv_rn(__ll2float_rn((long long)acc[i]) * kNormalUnfix, 3.0f);
}

__global__ void k_face_normals_backward(const float* __restrict__ V, const int32_t* __restrict__ F, int32_t nf,
                                        const float* __restrict__ dN, float* __restrict__ dV) {
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += gridDim.x * blockDim.x)
    face_normal_backward_one(V, F, f, dN, dV);
}

size_t normals_scratch_bytes(int32_t nv) { return align_up((size_t)nv * 3 * sizeof(unsigned long long), 256); }

void launch_vertex_normals(const float* V, int32_t nv, const int32_t* F, int32_t nf, float* N, void* scratch,
                           cudaStream_t s) {
  ProfScope ps("k_vertex_normals", s);
  unsigned long long* acc = (unsigned long long*)scratch;
  cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * 3 * (size_t)nv, s);
  const int blocks = (int)((nf + 255) / 256) < 4 * num_sms() ? (int)((nf + 255) / 256) : 4 * num_sms();
  k_face_normals_scatter<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(V, F, nf, acc);
  const int64_t n3 = 3 * (int64_t)nv;
  const int b2 = (int)((n3 + 255) / 256) < 4 * num_sms() ? (int)((n3 + 255) / 256) : 4 * num_sms();
  k_normals_finish<<<b2 > 0 ? b2 : 1, 256, 0, s>>>(acc, n3, N);
}

void launch_vertex_normals_backward(const float* V, int32_t nv, const int32_t* F, int32_t nf, const float* dN,
                                    float* dV, cudaStream_t s) {
  (void)nv;
  ProfScope ps("k_face_normals_backward", s);
  const int blocks = (int)((nf + 255) / 256) < 4 * num_sms() ? (int)((nf + 255) / 256) : 4 * num_sms();
  k_face_normals_backward<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(V, F, nf, dN, dV);
}

// ---------------------------------------------------------------------------
// LBVH build
// ---------------------------------------------------------------------------
// float <-> order-preserving unsigned, for atomicMin/Max on floats
__device__ __forceinline__ uint32_t f2ord(float f) {
  uint32_t b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float ord2f(uint32_t o) {
  return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

// scratch: bounds of the centroids as ordered uints [lo xyz, hi xyz]
__global__ void k_init_bounds(uint32_t* b) {
  if (threadIdx.x < 3) b[threadIdx.x] = 0xffffffffu;
  else if (threadIdx.x < 6) b[threadIdx.x] = 0u;
}

__device__ __forceinline__ float3 centroid_of(const float* V, const int32_t* F, int f) {
  const float3 v0 = load3(V + 3 * F[3 * f]), v1 = load3(V + 3 * F[3 * f + 1]), v2 = load3(V + 3 * F[3 * f + 2]);
  return (v0 + v1 + v2) * (1.0f / 3.0f);
}

__global__ void k_centroid_bounds(const float* __restrict__ V, const int32_t* __restrict__ F, int32_t nf,
                                  uint32_t* __restrict__ b) {
  float3 lo = mk(INFINITY, INFINITY, INFINITY), hi = mk(-INFINITY, -INFINITY, -INFINITY);
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += gridDim.x * blockDim.x) {
    const float3 c = centroid_of(V, F, f);
    lo = mk(fminf(lo.x, c.x), fminf(lo.y, c.y), fminf(lo.z, c.z));
    hi = mk(fmaxf(hi.x, c.x), fmaxf(hi.y, c.y), fmaxf(hi.z, c.z));
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo.x = fminf(lo.x, __shfl_xor_sync(kFull, lo.x, o));
    lo.y = fminf(lo.y, __shfl_xor_sync(kFull, lo.y, o));
    lo.z = fminf(lo.z, __shfl_xor_sync(kFull, lo.z, o));
    hi.x = fmaxf(hi.x, __shfl_xor_sync(kFull, hi.x, o));
    hi.y = fmaxf(hi.y, __shfl_xor_sync(kFull, hi.y, o));
    hi.z = fmaxf(hi.z, __shfl_xor_sync(kFull, hi.z, o));
  }
  if ((threadIdx.x & 31) == 0 && lo.x <= hi.x) {
    atomicMin(b + 0, f2ord(lo.x)); atomicMin(b + 1, f2ord(lo.y)); atomicMin(b + 2, f2ord(lo.z));
    atomicMax(b + 3, f2ord(hi.x)); atomicMax(b + 4, f2ord(hi.y)); atomicMax(b + 5, f2ord(hi.z));
  }
}

// 10 bits per axis interleaved into a 30-bit Morton code
__device__ __forceinline__ uint32_t spread10(uint32_t v) {
  v = (v | (v << 16)) & 0x030000FFu;
  v = (v | (v << 8)) & 0x0300F00Fu;
  v = (v | (v << 4)) & 0x030C30C3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

__global__ void k_morton(const float* __restrict__ V, const int32_t* __restrict__ F, int32_t nf,
                         const uint32_t* __restrict__ b, uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  const float3 lo = mk(ord2f(b[0]), ord2f(b[1]), ord2f(b[2]));
  const float3 hi = mk(ord2f(b[3]), ord2f(b[4]), ord2f(b[5]));
  const float3 ext = mk(fmaxf(hi.x - lo.x, 1e-30f), fmaxf(hi.y - lo.y, 1e-30f), fmaxf(hi.z - lo.z, 1e-30f));
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += gridDim.x * blockDim.x) {
    const float3 c = centroid_of(V, F, f);
    const uint32_t x = (uint32_t)fminf(fmaxf((c.x - lo.x) / ext.x * 1024.0f, 0.0f), 1023.0f);
    const uint32_t y = (uint32_t)fminf(fmaxf((c.y - lo.y) / ext.y * 1024.0f, 0.0f), 1023.0f);
    const uint32_t z = (uint32_t)fminf(fmaxf((c.z - lo.z) / ext.z * 1024.0f, 0.0f), 1023.0f);
    keys[f] = (spread10(x) << 2) | (spread10(y) << 1) | spread10(z);
    vals[f] = (uint32_t)f;
  }
}

// ---- stable LSD radix sort, 8 bits per pass -------------------------------
constexpr int kSortThreads = 256;
constexpr int kSortIpt = 4;
constexpr int kSortTile = kSortThreads * kSortIpt;
constexpr int kSortWarps = kSortThreads / 32;

// hist is digit-major: hist[d * nblocks + block]
__global__ void k_radix_hist(const uint32_t* __restrict__ keys, int32_t n, int shift, uint32_t* __restrict__ hist) {
  __shared__ uint32_t cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const int base = blockIdx.x * kSortTile;
  for (int j = 0; j < kSortIpt; ++j) {
    const int i = base + j * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 0xffu], 1u);
  }
  __syncthreads();
  hist[threadIdx.x * gridDim.x + blockIdx.x] = cnt[threadIdx.x];
}

// exclusive scan of m entries in one block of 1024 threads
__global__ void k_scan_exclusive(uint32_t* __restrict__ a, int32_t m) {
  __shared__ uint32_t part[1024];
  const int per = (m + 1023) / 1024;
  const int lo = threadIdx.x * per;
  const int hi = min(lo + per, m);
  uint32_t s = 0;
  for (int i = lo; i < hi; ++i) s += a[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {  // Hillis-Steele inclusive scan of the partial sums
    uint32_t v = threadIdx.x >= o ? part[threadIdx.x - o] : 0u;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  uint32_t run = threadIdx.x ? part[threadIdx.x - 1] : 0u;
  for (int i = lo; i < hi; ++i) {
    const uint32_t v = a[i];
    a[i] = run;
    run += v;
  }
}

// Scatter a tile keeping the input order among equal digits: items are taken
// in order j (stride kSortThreads), then warp, then lane; within a warp the
// rank among equal digits comes from __match_any_sync, across warps from a
// per-step prefix over per-warp digit counts.
__global__ void k_radix_scatter(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin, int32_t n,
                                int shift, const uint32_t* __restrict__ hist, uint32_t* __restrict__ kout,
                                uint32_t* __restrict__ vout) {
  __shared__ uint32_t off[256];
  __shared__ uint32_t wcnt[kSortWarps][256];
  __shared__ uint32_t step_total[256];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  off[tid] = hist[tid * gridDim.x + blockIdx.x];
  const int base = blockIdx.x * kSortTile;
  const unsigned lanemask_lt = (1u << lane) - 1u;
  for (int j = 0; j < kSortIpt; ++j) {
    for (int w = 0; w < kSortWarps; ++w) wcnt[w][tid] = 0;
    __syncthreads();
    const int i = base + j * kSortThreads + tid;
    const bool valid = i < n;
    uint32_t key = 0, val = 0, dg = 256;
    if (valid) {
      key = kin[i];
      val = vin[i];
      dg = (key >> shift) & 0xffu;
    }
    const unsigned peers = __match_any_sync(kFull, dg);
    const uint32_t rank = __popc(peers & lanemask_lt);
    if (valid && rank == 0) wcnt[warp][dg] = __popc(peers);
    __syncthreads();
    {  // thread tid owns digit tid: prefix over warps
      uint32_t run = 0;
      for (int w = 0; w < kSortWarps; ++w) {
        const uint32_t c = wcnt[w][tid];
        wcnt[w][tid] = run;
        run += c;
      }
      step_total[tid] = run;
    }
    __syncthreads();
    if (valid) {
      const uint32_t pos = off[dg] + wcnt[warp][dg] + rank;
      if (pos < (uint32_t)n) {
        kout[pos] = key;
        vout[pos] = val;
      }
    }
    __syncthreads();
    off[tid] += step_total[tid];
  }
}

// ---- Karras (2012) hierarchy ------------------------------------------------
// delta(a, b): length of the common prefix of keys a and b, with the index
// appended to break ties between equal keys; -1 outside [0, n).
__device__ __forceinline__ int lcp(const uint32_t* keys, int n, int a, int b) {
  if (b < 0 || b >= n) return -1;
  const uint32_t ka = keys[a], kb = keys[b];
  if (ka == kb) return 32 + __clz((uint32_t)a ^ (uint32_t)b);
  return __clz(ka ^ kb);
}

__global__ void k_karras(const uint32_t* __restrict__ keys, int32_t n, int2* __restrict__ bin_child,
                         int32_t* __restrict__ parent) {
  const int n_int = n - 1;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_int; i += gridDim.x * blockDim.x) {
    const int d = (lcp(keys, n, i, i + 1) - lcp(keys, n, i, i - 1)) >= 0 ? 1 : -1;
    const int dmin = lcp(keys, n, i, i - d);
    int lmax = 2;
    while (lcp(keys, n, i, i + lmax * d) > dmin) lmax *= 2;
    int l = 0;
    for (int t = lmax / 2; t >= 1; t /= 2)
      if (lcp(keys, n, i, i + (l + t) * d) > dmin) l += t;
    const int j = i + l * d;
    const int dnode = lcp(keys, n, i, j);
    int s = 0;
    for (int div = 2;; div *= 2) {
      const int t = (l + div - 1) / div;
      if (lcp(keys, n, i, i + (s + t) * d) > dnode) s += t;
      if (t <= 1) break;
    }
    const int gamma = i + s * d + (d < 0 ? -1 : 0);
    const int lo = min(i, j), hi = max(i, j);
    const int left = (lo == gamma) ? ~gamma : gamma;
    const int right = (hi == gamma + 1) ? ~(gamma + 1) : gamma + 1;
    bin_child[i] = make_int2(left, right);
    parent[left < 0 ? n_int + gamma : gamma] = i;
    parent[right < 0 ? n_int + gamma + 1 : gamma + 1] = i;
    if (i == 0) parent[0] = -1;
  }
}

// one triangle: a single internal node whose two children are both leaf 0
__global__ void k_single_leaf(int2* bin_child, int32_t* parent) {
  bin_child[0] = make_int2(~0, ~0);
  parent[0] = -1;
  parent[1] = 0;
}

__global__ void k_gather_leaf_tri(const uint32_t* __restrict__ vals, int32_t n, int32_t* __restrict__ leaf_tri) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) leaf_tri[i] = (int32_t)vals[i];
}

// ---- bottom-up bounds of the binary tree -----------------------------------
__device__ __forceinline__ void store_box(float4* box, float3 lo, float3 hi) {
  volatile float* b = reinterpret_cast<volatile float*>(box);
  b[0] = lo.x; b[1] = lo.y; b[2] = lo.z; b[3] = 0.f;
  b[4] = hi.x; b[5] = hi.y; b[6] = hi.z; b[7] = 0.f;
}

__device__ __forceinline__ void load_box(const float4* box, float3& lo, float3& hi) {
  const volatile float* b = reinterpret_cast<const volatile float*>(box);
  lo = mk(b[0], b[1], b[2]);
  hi = mk(b[4], b[5], b[6]);
}

// Each leaf writes its triangle record and box, then climbs: the first of two
// children to reach a node stops, the second merges both boxes, stores the
// node's box and goes on.  A path to the root has at most n_int nodes; the
// bound guards a corrupt tree.
__global__ void k_refit(const float* __restrict__ V, const int32_t* __restrict__ F, int32_t nf, BvhView B,
                        uint32_t* __restrict__ arrive) {
  const int n_int = B.hdr->n_int;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += gridDim.x * blockDim.x) {
    const int tri = B.leaf_tri[i];
    const float3 v0 = load3(V + 3 * F[3 * tri]), v1 = load3(V + 3 * F[3 * tri + 1]), v2 = load3(V + 3 * F[3 * tri + 2]);
    B.tris[3 * i + 0] = make_float4(v0.x, v0.y, v0.z, __int_as_float(tri));
    const float3 e1 = v1 - v0, e2 = v2 - v0;
    B.tris[3 * i + 1] = make_float4(e1.x, e1.y, e1.z, 0.f);
    B.tris[3 * i + 2] = make_float4(e2.x, e2.y, e2.z, 0.f);
    float3 lo = mk(fminf(v0.x, fminf(v1.x, v2.x)), fminf(v0.y, fminf(v1.y, v2.y)), fminf(v0.z, fminf(v1.z, v2.z)));
    float3 hi = mk(fmaxf(v0.x, fmaxf(v1.x, v2.x)), fmaxf(v0.y, fmaxf(v1.y, v2.y)), fmaxf(v0.z, fmaxf(v1.z, v2.z)));
    store_box(B.box_leaf + 2 * i, lo, hi);
    int me = ~i;
    int node = B.parent[n_int + i];
    for (int hops = 0; node >= 0 && node < n_int && hops <= n_int; ++hops) {
      const int2 ch = B.bin_child[node];
      const int sib = (ch.x == me) ? ch.y : ch.x;
      if (sib != kNoChild) {
        __threadfence();
        const uint32_t prev = atomicAdd(arrive + node, 1u);
        if (prev == 0) break;  // the sibling is still on its way
        __threadfence();
        float3 olo, ohi;
        load_box(sib >= 0 ? B.box_int + 2 * sib : B.box_leaf + 2 * (~sib), olo, ohi);
        lo = mk(fminf(lo.x, olo.x), fminf(lo.y, olo.y), fminf(lo.z, olo.z));
        hi = mk(fmaxf(hi.x, ohi.x), fmaxf(hi.y, ohi.y), fmaxf(hi.z, ohi.z));
      }
      store_box(B.box_int + 2 * node, lo, hi);
      me = node;
      node = B.parent[node];
    }
  }
}

// ---- binned SAH build (top-down) ---------------------------------------------
// A second builder of the same binary layout.  Top-down: each task is a
// contiguous range of a primitive permutation; its split is the bin boundary
// (of 32 centroid bins per axis; 16 in the warp builder) with the least
// surface area cost area(left box) * left count + area(right box) * right
// count, and the range
// is partitioned stably into [left | right].  Tasks larger than kSahSmall
// take four launches per tree level, each spread over chunks of kSahChunk
// positions so that the few huge tasks near the root use the whole GPU: bin
// (per-chunk shared-memory bins added into the task's bins), split (one warp
// per task), count (left primitives per chunk) and scatter (stable, each
// chunk at the offset of the chunks before it).  Smaller tasks are built
// down to their leaves by one warp each, in shared memory.  An internal node
// is numbered by its split position s (the last position of its left child),
// which is unique in [0, nf - 2]; the root's number is swapped with 0 so the
// root is node 0.  Splits deeper than kSahFreeDepth (large tasks) or
// kSahSmallFreeDepth (small ones) take the median, which bounds the depth
// (see launch_sah_topology).  Every decision is a deterministic function of
// the geometry: bins are integer sums, minima and maxima, and partitions are
// stable.
constexpr int kSahBins = 32;       // bins per axis of the large-task levels
constexpr int kSahSmallBins = 16;  // of the warp builder
constexpr int kSahTiny = 4;        // ranges up to this size split at the centroid median
constexpr int kSahSmall = 128;
constexpr int kSahFreeDepth = 24;
constexpr int kSahSmallFreeDepth = 56;
constexpr int kSahMaxLevels = 64;
constexpr int kSahChunk = 4096;
constexpr int kSahThreads = 256;
constexpr int kSahSmallWarps = 4;

struct SahTask {
  int a, n, parent, sd;       // range, parent node, side | depth << 1
  int chunk0, axis, bin, nl;  // first chunk of the level; the split (axis < 0: median)
  float4 lo, hi;              // binning bounds (xyz), a superset of the centroids
};
template <int kB>
struct SahBinsT {  // order-preserving uints for the float bounds
  uint32_t cnt[3][kB];
  uint32_t lo[3][kB][3];
  uint32_t hi[3][kB][3];
};
using SahBins = SahBinsT<kSahBins>;
using SahSmallBins = SahBinsT<kSahSmallBins>;
struct SahState {
  unsigned long long packed[kSahMaxLevels + 2];  // per level: tasks << 32 | chunks
  int n_small;
  int sroot;
};
struct SahView {
  float4* cen;
  float4* pbox;
  uint32_t* idx[2];
  SahTask* tasks[2];
  SahBins* bins[2];
  uint32_t* chunk_left;
  int4* small;  // (a, n, parent, side | depth << 1 | buffer << 30)
  SahState* st;
  int max_large, max_small, max_chunks;
};

template <int kB = kSahBins>
__device__ __forceinline__ int sah_bin(float c, float lo, float scale) {
  const int b = (int)__fmul_rn(__fsub_rn(c, lo), scale);
  return min(kB - 1, max(0, b));
}
template <int kB = kSahBins>
__device__ __forceinline__ float sah_scale(float lo, float hi) {
  const float ext = __fsub_rn(hi, lo);
  return ext > 0.0f ? __fdiv_rn((float)kB, ext) : 0.0f;
}
__device__ __forceinline__ float sah_area(float3 lo, float3 hi) {
  const float3 d = hi - lo;
  return d.x * d.y + d.y * d.z + d.z * d.x;
}
__device__ __forceinline__ int sah_split_id(int s, int sroot) { return s == sroot ? 0 : (s == 0 ? sroot : s); }
__device__ __forceinline__ void sah_set_child(BvhView& B, int node, int side, int ref) {
  reinterpret_cast<int*>(B.bin_child + node)[side] = ref;
}
__device__ __forceinline__ float comp(const float4& v, int k) { return k == 0 ? v.x : (k == 1 ? v.y : v.z); }
__device__ __forceinline__ float comp3(const float3& v, int k) { return k == 0 ? v.x : (k == 1 ? v.y : v.z); }

// primitive boxes and centroids, the identity permutation, bin_child cleared
// to kNoChild and internal parents to -1 (validation catches any link a build
// leaves unset, and the depth walks stop at an unset parent)
__global__ void k_sah_prims(const float* __restrict__ V, const int32_t* __restrict__ F, int32_t nf, SahView S,
                            BvhView B) {
  const int n_int = nf - 1;
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += gridDim.x * blockDim.x) {
    const float3 v0 = load3(V + 3 * F[3 * f]), v1 = load3(V + 3 * F[3 * f + 1]), v2 = load3(V + 3 * F[3 * f + 2]);
    const float3 c = (v0 + v1 + v2) * (1.0f / 3.0f);
    S.cen[f] = make_float4(c.x, c.y, c.z, 0.f);
    S.pbox[2 * f] =
        make_float4(fminf(v0.x, fminf(v1.x, v2.x)), fminf(v0.y, fminf(v1.y, v2.y)), fminf(v0.z, fminf(v1.z, v2.z)), 0.f);
    S.pbox[2 * f + 1] =
        make_float4(fmaxf(v0.x, fmaxf(v1.x, v2.x)), fmaxf(v0.y, fmaxf(v1.y, v2.y)), fmaxf(v0.z, fmaxf(v1.z, v2.z)), 0.f);
    S.idx[0][f] = (uint32_t)f;
    if (f < n_int) {
      B.bin_child[f] = make_int2(kNoChild, kNoChild);
      B.parent[f] = -1;
    }
  }
}

__device__ __forceinline__ int sah_chunks(int n) { return (n + kSahChunk - 1) / kSahChunk; }

// empty bins: zero counts, inverted bounds (threads i0, i0 + stride, ...)
template <int kB>
__device__ __forceinline__ void sah_zero_bins(SahBinsT<kB>* g, int i0, int stride) {
  uint32_t* cnt = &g->cnt[0][0];
  uint32_t* lo = &g->lo[0][0][0];
  uint32_t* hi = &g->hi[0][0][0];
  for (int i = i0; i < 3 * kB; i += stride) {
    cnt[i] = 0u;
    for (int q = 0; q < 3; ++q) {
      lo[3 * i + q] = 0xffffffffu;
      hi[3 * i + q] = 0u;
    }
  }
}

// the root task: large (level 0) or, for at most kSahSmall triangles, small
__global__ void k_sah_root(int32_t nf, const uint32_t* __restrict__ bounds, SahView S) {
  for (int i = threadIdx.x; i < kSahMaxLevels + 2; i += blockDim.x) S.st->packed[i] = 0ull;
  if (nf > kSahSmall) sah_zero_bins(&S.bins[0][0], threadIdx.x, blockDim.x);
  __syncthreads();
  if (threadIdx.x == 0) {
    S.st->sroot = -1;
    S.st->n_small = 0;
    if (nf > kSahSmall) {
      SahTask t;
      t.a = 0; t.n = nf; t.parent = -1; t.sd = 0;
      t.chunk0 = 0; t.axis = -1; t.bin = -1; t.nl = 0;
      t.lo = make_float4(ord2f(bounds[0]), ord2f(bounds[1]), ord2f(bounds[2]), 0.f);
      t.hi = make_float4(ord2f(bounds[3]), ord2f(bounds[4]), ord2f(bounds[5]), 0.f);
      S.tasks[0][0] = t;
      S.st->packed[0] = (1ull << 32) | (unsigned long long)sah_chunks(nf);
    } else {
      S.small[0] = make_int4(0, nf, -1, 0);
      S.st->n_small = 1;
    }
  }
}

template <int kB>
__device__ __forceinline__ void sah_flush(SahBinsT<kB>& sb, int k, int b, uint32_t n, float3 lo, float3 hi) {
  atomicAdd(&sb.cnt[k][b], n);
  atomicMin(&sb.lo[k][b][0], f2ord(lo.x)); atomicMin(&sb.lo[k][b][1], f2ord(lo.y)); atomicMin(&sb.lo[k][b][2], f2ord(lo.z));
  atomicMax(&sb.hi[k][b][0], f2ord(hi.x)); atomicMax(&sb.hi[k][b][1], f2ord(hi.y)); atomicMax(&sb.hi[k][b][2], f2ord(hi.z));
}

// best split of one axis from its bins: boundary i puts bins 0..i left
struct SahSplit {
  float cost;
  int axis, bin, nl;
  float3 llo, lhi, rlo, rhi;
};
template <int kB>
__device__ SahSplit sah_sweep(const SahBinsT<kB>& sb, int k) {
  SahSplit best;
  best.cost = INFINITY; best.axis = k; best.bin = -1; best.nl = 0;
  float rarea[kB];
  uint32_t rcnt[kB];
  float3 rl = mk(INFINITY, INFINITY, INFINITY), rh = mk(-INFINITY, -INFINITY, -INFINITY);
  uint32_t c = 0;
  for (int i = kB - 1; i >= 1; --i) {
    if (sb.cnt[k][i]) {
      rl = mk(fminf(rl.x, ord2f(sb.lo[k][i][0])), fminf(rl.y, ord2f(sb.lo[k][i][1])), fminf(rl.z, ord2f(sb.lo[k][i][2])));
      rh = mk(fmaxf(rh.x, ord2f(sb.hi[k][i][0])), fmaxf(rh.y, ord2f(sb.hi[k][i][1])), fmaxf(rh.z, ord2f(sb.hi[k][i][2])));
    }
    c += sb.cnt[k][i];
    rcnt[i] = c;
    rarea[i] = c ? sah_area(rl, rh) : 0.f;
  }
  float3 ll = mk(INFINITY, INFINITY, INFINITY), lh = mk(-INFINITY, -INFINITY, -INFINITY);
  uint32_t lc = 0;
  for (int i = 0; i < kB - 1; ++i) {
    if (sb.cnt[k][i]) {
      ll = mk(fminf(ll.x, ord2f(sb.lo[k][i][0])), fminf(ll.y, ord2f(sb.lo[k][i][1])), fminf(ll.z, ord2f(sb.lo[k][i][2])));
      lh = mk(fmaxf(lh.x, ord2f(sb.hi[k][i][0])), fmaxf(lh.y, ord2f(sb.hi[k][i][1])), fmaxf(lh.z, ord2f(sb.hi[k][i][2])));
    }
    lc += sb.cnt[k][i];
    const uint32_t rc = rcnt[i + 1];
    if (lc == 0 || rc == 0) continue;
    const float cost = sah_area(ll, lh) * (float)lc + rarea[i + 1] * (float)rc;
    if (cost < best.cost) {
      best.cost = cost; best.bin = i; best.nl = (int)lc;
      best.llo = ll; best.lhi = lh;
    }
  }
  if (best.bin >= 0) {  // the right box of the chosen boundary
    float3 a = mk(INFINITY, INFINITY, INFINITY), b = mk(-INFINITY, -INFINITY, -INFINITY);
    for (int i = best.bin + 1; i < kB; ++i)
      if (sb.cnt[k][i]) {
        a = mk(fminf(a.x, ord2f(sb.lo[k][i][0])), fminf(a.y, ord2f(sb.lo[k][i][1])), fminf(a.z, ord2f(sb.lo[k][i][2])));
        b = mk(fmaxf(b.x, ord2f(sb.hi[k][i][0])), fmaxf(b.y, ord2f(sb.hi[k][i][1])), fmaxf(b.z, ord2f(sb.hi[k][i][2])));
      }
    best.rlo = a; best.rhi = b;
  }
  return best;
}

// the task that owns chunk c (tasks are in chunk order: slot and chunks come
// from one 64-bit atomic)
__device__ __forceinline__ int sah_find_task(const SahTask* tasks, int ntask, int c) {
  int lo = 0, hi = ntask - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tasks[mid].chunk0 <= c) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

struct SahLevel {
  int ntask, nchunk;
};
__device__ __forceinline__ SahLevel sah_level(const SahView& S, int level) {
  const unsigned long long pk = S.st->packed[level];
  SahLevel l;
  l.ntask = min((int)(pk >> 32), S.max_large);
  l.nchunk = min((int)(pk & 0xffffffffull), S.max_chunks);
  return l;
}

__device__ __forceinline__ bool sah_free(const SahTask& T, float sc[3]) {
  sc[0] = sah_scale(T.lo.x, T.hi.x);
  sc[1] = sah_scale(T.lo.y, T.hi.y);
  sc[2] = sah_scale(T.lo.z, T.hi.z);
  return (T.sd >> 1) < kSahFreeDepth && (sc[0] > 0.f || sc[1] > 0.f || sc[2] > 0.f);
}

__device__ __forceinline__ bool sah_goes_left(const SahView& S, const SahTask& T, const float sc[3], uint32_t p, int i) {
  if (T.axis < 0) return i < T.nl;
  const float4 c = S.cen[p];
  return sah_bin(comp(c, T.axis), comp(T.lo, T.axis), sc[T.axis]) <= T.bin;
}

// 1/4 of a level: the bins of every task, chunk by chunk
__global__ void __launch_bounds__(kSahThreads) k_sah_bin(int level, SahView S) {
  __shared__ SahBins sb;
  const SahLevel L = sah_level(S, level);
  const SahTask* tasks = S.tasks[level & 1];
  const uint32_t* __restrict__ in = S.idx[level & 1];
  const int tid = threadIdx.x;
  for (int c = blockIdx.x; c < L.nchunk; c += gridDim.x) {
    const int t = sah_find_task(tasks, L.ntask, c);
    const SahTask T = tasks[t];
    float sc[3];
    if (!sah_free(T, sc)) continue;  // uniform over the block
    sah_zero_bins(&sb, tid, blockDim.x);
    __syncthreads();
    const int q0 = T.a + (c - T.chunk0) * kSahChunk, q1 = min(T.a + T.n, q0 + kSahChunk);
    // each thread bins a contiguous run, adding runs of equal bins at once
    const int run = (q1 - q0 + blockDim.x - 1) / blockDim.x;
    const int p0 = q0 + tid * run, p1 = min(q1, p0 + run);
    int cb[3] = {-1, -1, -1};
    uint32_t cn[3] = {0u, 0u, 0u};
    float3 clo[3], chi[3];
    for (int pos = p0; pos < p1; ++pos) {
      const uint32_t p = in[pos];
      const float4 c4 = S.cen[p], lo = S.pbox[2 * p], hi = S.pbox[2 * p + 1];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        if (sc[k] <= 0.f) continue;
        const int b = sah_bin(comp(c4, k), comp(T.lo, k), sc[k]);
        if (b != cb[k]) {
          if (cb[k] >= 0) sah_flush(sb, k, cb[k], cn[k], clo[k], chi[k]);
          cb[k] = b; cn[k] = 0u;
          clo[k] = mk(INFINITY, INFINITY, INFINITY);
          chi[k] = mk(-INFINITY, -INFINITY, -INFINITY);
        }
        ++cn[k];
        clo[k] = mk(fminf(clo[k].x, lo.x), fminf(clo[k].y, lo.y), fminf(clo[k].z, lo.z));
        chi[k] = mk(fmaxf(chi[k].x, hi.x), fmaxf(chi[k].y, hi.y), fmaxf(chi[k].z, hi.z));
      }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k)
      if (cb[k] >= 0) sah_flush(sb, k, cb[k], cn[k], clo[k], chi[k]);
    __syncthreads();
    SahBins& G = S.bins[level & 1][t];
    for (int i = tid; i < 3 * kSahBins; i += blockDim.x) {
      const int k = i / kSahBins, b = i % kSahBins;
      if (!sb.cnt[k][b]) continue;
      atomicAdd(&G.cnt[k][b], sb.cnt[k][b]);
      for (int q = 0; q < 3; ++q) {
        atomicMin(&G.lo[k][b][q], sb.lo[k][b][q]);
        atomicMax(&G.hi[k][b][q], sb.hi[k][b][q]);
      }
    }
    __syncthreads();
  }
}

// 2/4: one warp per task chooses the split, numbers the node, links it to
// its parent and queues the children (large ones for the next level with
// cleared bins, the rest for the warp builder)
__global__ void __launch_bounds__(128) k_sah_split(int level, SahView S, BvhView B) {
  const SahLevel L = sah_level(S, level);
  SahTask* tasks = S.tasks[level & 1];
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  for (int t = gw; t < L.ntask; t += nw) {
    SahTask T = tasks[t];
    const int depth = T.sd >> 1;
    float sc[3];
    int axis = -1, bin = -1, nl = T.n / 2;
    float3 llo = mk(T.lo.x, T.lo.y, T.lo.z), lhi = mk(T.hi.x, T.hi.y, T.hi.z), rlo = llo, rhi = lhi;
    if (sah_free(T, sc)) {
      const SahBins& G = S.bins[level & 1][t];
      SahSplit sp;
      sp.cost = INFINITY; sp.bin = -1; sp.axis = lane; sp.nl = 0;
      if (lane < 3 && sc[lane] > 0.f) sp = sah_sweep(G, lane);
      float bc = INFINITY;
      for (int k = 0; k < 3; ++k) {
        const float ck = __shfl_sync(kFull, sp.cost, k);
        const int bk = __shfl_sync(kFull, sp.bin, k);
        if (bk >= 0 && ck < bc) { bc = ck; axis = k; }
      }
      if (axis >= 0) {
        bin = __shfl_sync(kFull, sp.bin, axis);
        nl = __shfl_sync(kFull, sp.nl, axis);
        llo = mk(__shfl_sync(kFull, sp.llo.x, axis), __shfl_sync(kFull, sp.llo.y, axis), __shfl_sync(kFull, sp.llo.z, axis));
        lhi = mk(__shfl_sync(kFull, sp.lhi.x, axis), __shfl_sync(kFull, sp.lhi.y, axis), __shfl_sync(kFull, sp.lhi.z, axis));
        rlo = mk(__shfl_sync(kFull, sp.rlo.x, axis), __shfl_sync(kFull, sp.rlo.y, axis), __shfl_sync(kFull, sp.rlo.z, axis));
        rhi = mk(__shfl_sync(kFull, sp.rhi.x, axis), __shfl_sync(kFull, sp.rhi.y, axis), __shfl_sync(kFull, sp.rhi.z, axis));
      }
    }
    int child_slot[2] = {-1, -1};
    if (lane == 0) {
      tasks[t].axis = axis;
      tasks[t].bin = bin;
      tasks[t].nl = nl;
      const int s = T.a + nl - 1;
      int sroot;
      if (T.parent < 0) {
        sroot = s;
        S.st->sroot = s;
      } else {
        sroot = S.st->sroot;
      }
      const int id = sah_split_id(s, sroot);
      B.parent[id] = T.parent;
      if (T.parent >= 0) sah_set_child(B, T.parent, T.sd & 1, id);
      for (int c = 0; c < 2; ++c) {
        const int ca = c ? T.a + nl : T.a, cn = c ? T.n - nl : nl;
        if (cn <= kSahSmall) {  // (one triangle: the warp builder writes the leaf)
          const int slot = atomicAdd(&S.st->n_small, 1);
          if (slot < S.max_small) S.small[slot] = make_int4(ca, cn, id, c | ((depth + 1) << 1) | (((level + 1) & 1) << 30));
          else atomicExch(&B.hdr->corrupt, 1);  // more tasks than disjoint ranges: never expected
        } else {
          const unsigned long long old =
              atomicAdd(&S.st->packed[level + 1], (1ull << 32) | (unsigned long long)sah_chunks(cn));
          const int slot = (int)(old >> 32), chunk0 = (int)(old & 0xffffffffull);
          if (slot < S.max_large && chunk0 + sah_chunks(cn) <= S.max_chunks) {
            SahTask ct;
            ct.a = ca; ct.n = cn; ct.parent = id; ct.sd = c | ((depth + 1) << 1);
            ct.chunk0 = chunk0; ct.axis = -1; ct.bin = -1; ct.nl = 0;
            const float3 lo = c ? rlo : llo, hi = c ? rhi : lhi;
            ct.lo = make_float4(lo.x, lo.y, lo.z, 0.f);
            ct.hi = make_float4(hi.x, hi.y, hi.z, 0.f);
            S.tasks[(level + 1) & 1][slot] = ct;
            child_slot[c] = slot;
          } else {
            atomicExch(&B.hdr->corrupt, 1);
          }
        }
      }
    }
    for (int c = 0; c < 2; ++c) {
      const int slot = __shfl_sync(kFull, child_slot[c], 0);
      if (slot >= 0) sah_zero_bins(&S.bins[(level + 1) & 1][slot], lane, 32);
    }
  }
}

// 3/4: left primitives of every chunk
__global__ void __launch_bounds__(kSahThreads) k_sah_count(int level, SahView S) {
  __shared__ int s_sum;
  const SahLevel L = sah_level(S, level);
  const SahTask* tasks = S.tasks[level & 1];
  const uint32_t* __restrict__ in = S.idx[level & 1];
  for (int c = blockIdx.x; c < L.nchunk; c += gridDim.x) {
    const SahTask T = tasks[sah_find_task(tasks, L.ntask, c)];
    float sc[3];
    sah_free(T, sc);
    if (threadIdx.x == 0) s_sum = 0;
    __syncthreads();
    const int i0 = (c - T.chunk0) * kSahChunk, i1 = min(T.n, i0 + kSahChunk);
    int cnt = 0;
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) cnt += sah_goes_left(S, T, sc, in[T.a + i], i) ? 1 : 0;
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(kFull, cnt, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&s_sum, cnt);
    __syncthreads();
    if (threadIdx.x == 0) S.chunk_left[c] = (uint32_t)s_sum;
    __syncthreads();
  }
}

// 4/4: stable scatter of every chunk to [left | right] of its task
__global__ void __launch_bounds__(kSahThreads) k_sah_scatter(int level, SahView S, BvhView B) {
  __shared__ uint32_t s_warp[kSahThreads / 32];
  __shared__ int s_prefix;
  const SahLevel L = sah_level(S, level);
  const SahTask* tasks = S.tasks[level & 1];
  const uint32_t* __restrict__ in = S.idx[level & 1];
  uint32_t* out = S.idx[(level + 1) & 1];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int c = blockIdx.x; c < L.nchunk; c += gridDim.x) {
    const SahTask T = tasks[sah_find_task(tasks, L.ntask, c)];
    float sc[3];
    sah_free(T, sc);
    if (tid == 0) s_prefix = 0;
    __syncthreads();
    int pre = 0;
    for (int j = T.chunk0 + tid; j < c; j += blockDim.x) pre += (int)S.chunk_left[j];
    for (int o = 16; o > 0; o >>= 1) pre += __shfl_xor_sync(kFull, pre, o);
    if (lane == 0 && pre) atomicAdd(&s_prefix, pre);
    __syncthreads();
    const int i0 = (c - T.chunk0) * kSahChunk, i1 = min(T.n, i0 + kSahChunk);
    int lbase = s_prefix, rbase = i0 - s_prefix;
    for (int base = i0; base < i1; base += blockDim.x) {
      const int i = base + tid;
      const bool valid = i < i1;
      uint32_t p = 0u;
      bool left = false;
      if (valid) {
        p = in[T.a + i];
        left = sah_goes_left(S, T, sc, p, i);
      }
      const unsigned bal = __ballot_sync(kFull, left);
      if (lane == 0) s_warp[wid] = __popc(bal);
      __syncthreads();
      int woff = 0, tot = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        const int cw = (int)s_warp[w];
        if (w < wid) woff += cw;
        tot += cw;
      }
      const int lrank = woff + __popc(bal & ((1u << lane) - 1u));
      if (valid) {  // positions stay inside the task even if bins and partition disagreed
        const int q = left ? lbase + lrank : T.nl + rbase + (i - base - lrank);
        if (q < T.n) out[T.a + q] = p;
      }
      lbase += tot;
      rbase += min((int)blockDim.x, i1 - base) - tot;
      __syncthreads();
    }
    if (tid == 0 && i1 == T.n && lbase != T.nl) atomicExch(&B.hdr->corrupt, 1);  // never expected
  }
}

// Small tasks: one warp builds a whole subtree (at most kSahSmall triangles)
// with the same binned SAH, the range held in shared memory.
__global__ void __launch_bounds__(32 * kSahSmallWarps) k_sah_small(SahView S, BvhView B) {
  __shared__ uint32_t s_ids[kSahSmallWarps][kSahSmall], s_tmp[kSahSmallWarps][kSahSmall];
  __shared__ int4 s_stack[kSahSmallWarps][kSahSmall / 2 + 1];
  __shared__ SahSmallBins s_bins[kSahSmallWarps];
  const int n_int = B.hdr->n_int;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t* ids = s_ids[w];
  uint32_t* tmp = s_tmp[w];
  int4* stack = s_stack[w];
  SahSmallBins& sb = s_bins[w];
  const int nsmall = min(S.st->n_small, S.max_small);
  for (int t = blockIdx.x * kSahSmallWarps + w; t < nsmall; t += gridDim.x * kSahSmallWarps) {
    const int4 T = S.small[t];
    const int a = T.x, n = T.y;
    const uint32_t* in = S.idx[(T.w >> 30) & 1];
    if (n == 1) {  // a one-triangle child of a large task
      if (lane == 0) {
        sah_set_child(B, T.z, T.w & 1, ~a);
        B.parent[n_int + a] = T.z;
        B.leaf_tri[a] = (int32_t)in[a];
      }
      continue;
    }
    for (int i = lane; i < n; i += 32) ids[i] = in[a + i];
    int sroot = T.z < 0 ? -1 : S.st->sroot;
    int sp = 0;
    if (lane == 0) stack[0] = make_int4(0, n, T.z, T.w & 0x3fffffff);
    sp = 1;
    __syncwarp();
    while (sp > 0) {
      --sp;
      const int4 e = stack[sp];
      __syncwarp();
      const int ra = e.x, rn = e.y, par = e.z, side = e.w & 1, depth = e.w >> 1;
      // centroid bounds of the range
      float3 lo = mk(INFINITY, INFINITY, INFINITY), hi = mk(-INFINITY, -INFINITY, -INFINITY);
      for (int i = lane; i < rn; i += 32) {
        const float4 c = S.cen[ids[ra + i]];
        lo = mk(fminf(lo.x, c.x), fminf(lo.y, c.y), fminf(lo.z, c.z));
        hi = mk(fmaxf(hi.x, c.x), fmaxf(hi.y, c.y), fmaxf(hi.z, c.z));
      }
      for (int o = 16; o > 0; o >>= 1) {
        lo.x = fminf(lo.x, __shfl_xor_sync(kFull, lo.x, o));
        lo.y = fminf(lo.y, __shfl_xor_sync(kFull, lo.y, o));
        lo.z = fminf(lo.z, __shfl_xor_sync(kFull, lo.z, o));
        hi.x = fmaxf(hi.x, __shfl_xor_sync(kFull, hi.x, o));
        hi.y = fmaxf(hi.y, __shfl_xor_sync(kFull, hi.y, o));
        hi.z = fmaxf(hi.z, __shfl_xor_sync(kFull, hi.z, o));
      }
      const float sc[3] = {sah_scale<kSahSmallBins>(lo.x, hi.x), sah_scale<kSahSmallBins>(lo.y, hi.y),
                           sah_scale<kSahSmallBins>(lo.z, hi.z)};
      int axis = -1, bin = -1, nl = rn / 2;
      // a range of at most kSahTiny triangles splits at the median of its
      // centroids along their longest extent (ties by position): binning
      // would cost far more than it can gain on a handful of triangles
      const bool tiny = rn <= kSahTiny;
      int tiny_rank = 0;
      if (tiny) {
        const float3 ext = hi - lo;
        const int la = (ext.x >= ext.y && ext.x >= ext.z) ? 0 : (ext.y >= ext.z ? 1 : 2);
        const float c = lane < rn ? comp(S.cen[ids[ra + lane]], la) : 0.f;
        for (int j = 0; j < rn; ++j) {
          const float cj = __shfl_sync(kFull, c, j);
          tiny_rank += (cj < c || (cj == c && j < (int)lane)) ? 1 : 0;
        }
      } else if (depth < kSahSmallFreeDepth && (sc[0] > 0.f || sc[1] > 0.f || sc[2] > 0.f)) {
        sah_zero_bins(&sb, lane, 32);
        __syncwarp();
        for (int i = lane; i < rn; i += 32) {
          const uint32_t p = ids[ra + i];
          const float4 c = S.cen[p], plo = S.pbox[2 * p], phi = S.pbox[2 * p + 1];
          for (int k = 0; k < 3; ++k) {
            if (sc[k] <= 0.f) continue;
            sah_flush(sb, k, sah_bin<kSahSmallBins>(comp(c, k), comp3(lo, k), sc[k]), 1u, mk(plo.x, plo.y, plo.z),
                      mk(phi.x, phi.y, phi.z));
          }
        }
        __syncwarp();
        SahSplit sp3;
        sp3.cost = INFINITY; sp3.bin = -1; sp3.axis = lane; sp3.nl = 0;
        if (lane < 3 && sc[lane] > 0.f) sp3 = sah_sweep(sb, lane);
        float bc = INFINITY;
        for (int k = 0; k < 3; ++k) {
          const float ck = __shfl_sync(kFull, sp3.cost, k);
          const int bk = __shfl_sync(kFull, sp3.bin, k);
          if (bk >= 0 && ck < bc) { bc = ck; axis = k; }
        }
        if (axis >= 0) {
          bin = __shfl_sync(kFull, sp3.bin, axis);
          nl = __shfl_sync(kFull, sp3.nl, axis);
        }
        __syncwarp();
      }
      // stable partition of ids[ra, ra + rn) through tmp
      int lbase = 0;
      int rbase = 0;
      for (int base = 0; base < rn; base += 32) {
        const int i = base + lane;
        const bool valid = i < rn;
        uint32_t p = 0u;
        bool left = false;
        if (valid) {
          p = ids[ra + i];
          left = tiny ? tiny_rank < nl
                      : (axis >= 0 ? sah_bin<kSahSmallBins>(comp(S.cen[p], axis), comp3(lo, axis), sc[axis]) <= bin
                                   : i < nl);
        }
        const unsigned bal = __ballot_sync(kFull, left);
        const int lr = __popc(bal & ((1u << lane) - 1u));
        if (valid) {  // inside the range even if bins and partition disagreed
          const int q = left ? lbase + lr : nl + rbase + (lane - lr);
          if (q < rn) tmp[ra + q] = p;
        }
        const int tot = __popc(bal);
        lbase += tot;
        rbase += min(32, rn - base) - tot;
      }
      __syncwarp();
      for (int i = lane; i < rn; i += 32) ids[ra + i] = tmp[ra + i];
      __syncwarp();
      if (lbase != nl && lane == 0) atomicExch(&B.hdr->corrupt, 1);
      const int s = a + ra + nl - 1;
      if (par < 0) sroot = s;  // the whole tree is this one task
      const int id = sah_split_id(s, sroot);
      if (lane == 0) {
        B.parent[id] = par;
        if (par >= 0) sah_set_child(B, par, side, id);
        if (par < 0) S.st->sroot = s;
      }
      for (int c = 1; c >= 0; --c) {
        const int ca = c ? ra + nl : ra, cn = c ? rn - nl : nl;
        if (cn == 1) {
          if (lane == 0) {
            sah_set_child(B, id, c, ~(a + ca));
            B.parent[n_int + a + ca] = id;
          }
        } else {
          if (lane == 0) stack[sp] = make_int4(ca, cn, id, c | ((depth + 1) << 1));
          ++sp;
        }
      }
      __syncwarp();
    }
    for (int i = lane; i < n; i += 32) B.leaf_tri[a + i] = (int32_t)ids[i];
    __syncwarp();
  }
}

// ---- the 4-wide BVH ----------------------------------------------------------
// flag[j] = 1 when binary node j sits at even depth (walks up to the root)
__global__ void k_even_depth(BvhView B, uint32_t* __restrict__ flag) {
  const int n_int = B.hdr->n_int;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n_int; j += gridDim.x * blockDim.x) {
    int d = 0, p = j;
    for (int hops = 0; hops <= n_int && p > 0; ++hops) {
      p = B.parent[p];
      ++d;
    }
    flag[j] = (d & 1) ? 0u : 1u;
  }
}

// after an exclusive scan of the flags: node4 index per even-depth node, -1 else
__global__ void k_bin_to4(BvhView B, const uint32_t* __restrict__ scanned) {
  const int n_int = B.hdr->n_int;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n_int; j += gridDim.x * blockDim.x) {
    int d = 0, p = j;
    for (int hops = 0; hops <= n_int && p > 0; ++hops) {
      p = B.parent[p];
      ++d;
    }
    B.bin_to4[j] = (d & 1) ? -1 : (int)scanned[j];
    if (j == n_int - 1) B.hdr->n4 = (int)scanned[j] + ((d & 1) ? 0 : 1);
  }
}

// children of 4-wide node bin_to4[j] = the grandchildren of binary node j (a
// leaf child stays as it is); refs in row 6, binary sources in row 7
__global__ void k_node4_topology(BvhView B) {
  const int n_int = B.hdr->n_int;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n_int; j += gridDim.x * blockDim.x) {
    const int m = B.bin_to4[j];
    if (m < 0) continue;
    int ref[4] = {kNoChild, kNoChild, kNoChild, kNoChild};
    int srcs[4] = {kNoChild, kNoChild, kNoChild, kNoChild};
    int k = 0;
    const int2 ch = B.bin_child[j];
    const int c2[2] = {ch.x, ch.y};
    for (int a = 0; a < 2; ++a) {
      const int c = c2[a];
      if (c == kNoChild) continue;
      if (c < 0) {
        ref[k] = c; srcs[k] = c; ++k;
        continue;
      }
      const int2 g = B.bin_child[c];
      const int gg[2] = {g.x, g.y};
      for (int b = 0; b < 2; ++b) {
        const int x = gg[b];
        if (x == kNoChild) continue;
        ref[k] = x < 0 ? x : B.bin_to4[x];
        srcs[k] = x;
        ++k;
      }
    }
    reinterpret_cast<int4*>(B.node4)[8 * m + 6] = make_int4(ref[0], ref[1], ref[2], ref[3]);
    reinterpret_cast<int4*>(B.node4)[8 * m + 7] = make_int4(srcs[0], srcs[1], srcs[2], srcs[3]);
  }
}

// child boxes of every 4-wide node from the binary boxes (after each refit)
__global__ void k_node4_boxes(BvhView B) {
  const int n4 = B.hdr->n4;
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n4; m += gridDim.x * blockDim.x) {
    const int4 sv = reinterpret_cast<const int4*>(B.node4)[8 * m + 7];
    const int srcs[4] = {sv.x, sv.y, sv.z, sv.w};
    float r[6][4];
    for (int k = 0; k < 4; ++k) {
      float3 lo = mk(INFINITY, INFINITY, INFINITY), hi = mk(-INFINITY, -INFINITY, -INFINITY);
      const int x = srcs[k];
      if (x != kNoChild) {
        const float4* bx = x >= 0 ? B.box_int + 2 * x : B.box_leaf + 2 * (~x);
        const float4 a = bx[0], b = bx[1];
        lo = mk(a.x, a.y, a.z);
        hi = mk(b.x, b.y, b.z);
      }
      r[0][k] = lo.x; r[1][k] = hi.x; r[2][k] = lo.y; r[3][k] = hi.y; r[4][k] = lo.z; r[5][k] = hi.z;
    }
    for (int row = 0; row < 6; ++row) B.node4[8 * m + row] = make_float4(r[row][0], r[row][1], r[row][2], r[row][3]);
  }
}

// binary nodes for the 2-wide traversal, from the binary boxes (after each refit)
__global__ void k_node2_boxes(BvhView B) {
  const int n_int = B.hdr->n_int;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n_int; j += gridDim.x * blockDim.x) {
    const int2 ch = B.bin_child[j];
    float3 lo[2], hi[2];
    const int c2[2] = {ch.x, ch.y};
    for (int k = 0; k < 2; ++k) {
      lo[k] = mk(INFINITY, INFINITY, INFINITY);
      hi[k] = mk(-INFINITY, -INFINITY, -INFINITY);
      const int x = c2[k];
      if (x != kNoChild) {
        const float4* bx = x >= 0 ? B.box_int + 2 * x : B.box_leaf + 2 * (~x);
        const float4 a = bx[0], b = bx[1];
        lo[k] = mk(a.x, a.y, a.z);
        hi[k] = mk(b.x, b.y, b.z);
      }
    }
    B.node2[4 * j + 0] = make_float4(lo[0].x, hi[0].x, lo[0].y, hi[0].y);
    B.node2[4 * j + 1] = make_float4(lo[1].x, hi[1].x, lo[1].y, hi[1].y);
    B.node2[4 * j + 2] = make_float4(lo[0].z, hi[0].z, lo[1].z, hi[1].z);
    reinterpret_cast<int4*>(B.node2)[4 * j + 3] = make_int4(ch.x, ch.y, 0, 0);
  }
}

// Validation of the built hierarchy: every reference in range, every parent
// link consistent with the child lists.  The traversal reads `corrupt` once
// and refuses to run on a tree that failed.
__global__ void k_validate(BvhView B) {
  const int n_int = B.hdr->n_int, n4 = B.hdr->n4, nf = B.hdr->nf;
  bool bad = (n4 < 1 || n4 > n_int);
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n_int; j += gridDim.x * blockDim.x) {
    const int2 ch = B.bin_child[j];
    const int c2[2] = {ch.x, ch.y};
    for (int k = 0; k < 2; ++k) {
      const int c = c2[k];
      if (c >= 0) bad |= c >= n_int || B.parent[c] != j;
      else bad |= (uint32_t)(~c) >= (uint32_t)nf || (nf > 1 && B.parent[n_int + ~c] != j);
    }
    if (j < n4) {
      const int4 r = reinterpret_cast<const int4*>(B.node4)[8 * j + 6];
      const int rr[4] = {r.x, r.y, r.z, r.w};
      for (int k = 0; k < 4; ++k) {
        const int c = rr[k];
        if (c == kNoChild) continue;
        bad |= c >= 0 ? c >= n4 : (uint32_t)(~c) >= (uint32_t)nf;
      }
    }
  }
  if (bad) atomicExch(&B.hdr->corrupt, 1);
}

__global__ void k_bvh_header(BvhHeader* h, int32_t nf) {
  h->nf = nf;
  h->n_int = nf > 1 ? nf - 1 : 1;
  h->n4 = 0;
  h->corrupt = 0;
}

// scratch layout for build/refit
struct BuildScratch {
  uint32_t *keys_a, *keys_b, *vals_a, *vals_b, *hist, *arrive, *bounds;
  SahView sah;
  size_t total;
  BuildScratch(void* base, int32_t nf) {
    const int nblocks = (nf + kSortTile - 1) / kSortTile;
    const size_t n_int = nf > 1 ? (size_t)nf - 1 : 1;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o = align_up(o + bytes, 256); return r; };
    const size_t ka = take(sizeof(uint32_t) * nf), kb = take(sizeof(uint32_t) * nf);
    const size_t va = take(sizeof(uint32_t) * nf), vb = take(sizeof(uint32_t) * nf);
    const size_t hi = take(sizeof(uint32_t) * 256 * (size_t)nblocks);
    const size_t ar = take(sizeof(uint32_t) * n_int);
    const size_t bo = take(sizeof(uint32_t) * 8);
    // binned SAH build: centroids, boxes, task lists and bins of two levels,
    // left counts per chunk, small tasks
    sah.max_large = nf / (kSahSmall + 1) + 1;
    sah.max_small = nf + 1;
    sah.max_chunks = nf / kSahChunk + sah.max_large + 1;
    const size_t ce = take(sizeof(float4) * nf), pb = take(sizeof(float4) * 2 * (size_t)nf);
    const size_t t0 = take(sizeof(SahTask) * sah.max_large), t1 = take(sizeof(SahTask) * sah.max_large);
    const size_t b0 = take(sizeof(SahBins) * sah.max_large), b1 = take(sizeof(SahBins) * sah.max_large);
    const size_t cl = take(sizeof(uint32_t) * sah.max_chunks);
    const size_t sm = take(sizeof(int4) * sah.max_small), st = take(sizeof(SahState));
    total = o;
    char* b = (char*)base;
    keys_a = (uint32_t*)(b + ka); keys_b = (uint32_t*)(b + kb);
    vals_a = (uint32_t*)(b + va); vals_b = (uint32_t*)(b + vb);
    hist = (uint32_t*)(b + hi); arrive = (uint32_t*)(b + ar); bounds = (uint32_t*)(b + bo);
    sah.cen = (float4*)(b + ce);
    sah.pbox = (float4*)(b + pb);
    sah.idx[0] = vals_a;
    sah.idx[1] = vals_b;
    sah.tasks[0] = (SahTask*)(b + t0);
    sah.tasks[1] = (SahTask*)(b + t1);
    sah.bins[0] = (SahBins*)(b + b0);
    sah.bins[1] = (SahBins*)(b + b1);
    sah.chunk_left = (uint32_t*)(b + cl);
    sah.small = (int4*)(b + sm);
    sah.st = (SahState*)(b + st);
  }
};

size_t bvh_scratch_bytes(int32_t nf) { return BuildScratch(nullptr, nf).total; }

static int grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  const int64_t cap = 8 * (int64_t)num_sms();
  if (b > cap) b = cap;
  return b < 1 ? 1 : (int)b;
}

void launch_refit(const float* V, const int32_t* F, int32_t nf, void* bvh, void* scratch, cudaStream_t s) {
  BvhView B = bvh_view(bvh, nf);
  BuildScratch S(scratch, nf);
  const size_t n_int = nf > 1 ? (size_t)nf - 1 : 1;
  ProfScope ps("k_refit", s);
  cudaMemsetAsync(S.arrive, 0, sizeof(uint32_t) * n_int, s);
  k_refit<<<grid_for(nf, 256), 256, 0, s>>>(V, F, nf, B, S.arrive);
  k_node2_boxes<<<grid_for((int64_t)n_int, 256), 256, 0, s>>>(B);
  k_node4_boxes<<<grid_for((int64_t)n_int, 256), 256, 0, s>>>(B);
}

// Binned SAH topology (see above).  Large levels: kSahFreeDepth levels of
// free splits, then median splits, which halve a task per level, so after
// ceil(log2(nf / kSahSmall)) + 1 more levels every task is small; small
// tasks take free splits to depth kSahSmallFreeDepth, then at most
// log2(kSahSmall) median levels: the tree is at most 63 deep, within the
// traversal's 64-entry stack.  Levels beyond the last large one launch and
// return at once (the host does not wait to learn how many there were).
static void launch_sah_topology(const float* V, const int32_t* F, int32_t nf, BvhView& B, BuildScratch& S,
                                cudaStream_t s) {
  k_sah_prims<<<grid_for(nf, 256), 256, 0, s>>>(V, F, nf, S.sah, B);
  k_sah_root<<<1, 64, 0, s>>>(nf, S.bounds, S.sah);
  int levels = 0;
  if (nf > kSahSmall) {
    int lg = 0;
    while (((int64_t)kSahSmall << lg) < (int64_t)nf) ++lg;
    levels = kSahFreeDepth + lg + 2;
    if (levels > kSahMaxLevels) levels = kSahMaxLevels;
  }
  const int grid = 4 * num_sms();
  {
    ProfScope ps("sah_large_levels", s);
    for (int L = 0; L < levels; ++L) {
      k_sah_bin<<<grid, kSahThreads, 0, s>>>(L, S.sah);
      k_sah_split<<<grid_for(S.sah.max_large * 32, 128), 128, 0, s>>>(L, S.sah, B);
      k_sah_count<<<grid, kSahThreads, 0, s>>>(L, S.sah);
      k_sah_scatter<<<grid, kSahThreads, 0, s>>>(L, S.sah, B);
    }
  }
  ProfScope ps("sah_small", s);
  k_sah_small<<<grid_for(nf / 2 + 1, 32 * kSahSmallWarps), 32 * kSahSmallWarps, 0, s>>>(S.sah, B);
}

// Exclusive scan of m entries in place (one CTA; used by the mesh topology).
void launch_scan_exclusive(uint32_t* a, int32_t m, cudaStream_t s) { k_scan_exclusive<<<1, 1024, 0, s>>>(a, m); }

void launch_build(const float* V, const int32_t* F, int32_t nf, void* bvh, void* scratch, cudaStream_t s) {
  BvhView B = bvh_view(bvh, nf);
  BuildScratch S(scratch, nf);
  const int n_int = nf > 1 ? nf - 1 : 1;
  const bool sah = g_tuning.bvh_builder == 1 && nf > 1;
  {
    ProfScope ps(sah ? "sah_build" : "lbvh_build", s);
    k_bvh_header<<<1, 1, 0, s>>>(B.hdr, nf);
    k_init_bounds<<<1, 32, 0, s>>>(S.bounds);
    k_centroid_bounds<<<grid_for(nf, 256), 256, 0, s>>>(V, F, nf, S.bounds);
    if (sah) {
      launch_sah_topology(V, F, nf, B, S, s);
    } else {
      k_morton<<<grid_for(nf, 256), 256, 0, s>>>(V, F, nf, S.bounds, S.keys_a, S.vals_a);
      const int nblocks = (nf + kSortTile - 1) / kSortTile;
      uint32_t *kin = S.keys_a, *vin = S.vals_a, *kout = S.keys_b, *vout = S.vals_b;
      for (int shift = 0; shift < 32; shift += 8) {
        k_radix_hist<<<nblocks, kSortThreads, 0, s>>>(kin, nf, shift, S.hist);
        k_scan_exclusive<<<1, 1024, 0, s>>>(S.hist, 256 * nblocks);
        k_radix_scatter<<<nblocks, kSortThreads, 0, s>>>(kin, vin, nf, shift, S.hist, kout, vout);
        uint32_t* t = kin; kin = kout; kout = t;
        t = vin; vin = vout; vout = t;
      }
      // after an even number of passes the sorted data is back in keys_a/vals_a
      k_gather_leaf_tri<<<grid_for(nf, 256), 256, 0, s>>>(vin, nf, B.leaf_tri);
      if (nf > 1) {
        k_karras<<<grid_for(nf - 1, 256), 256, 0, s>>>(kin, nf, B.bin_child, B.parent);
      } else {
        k_single_leaf<<<1, 1, 0, s>>>(B.bin_child, B.parent);
      }
    }
    // 4-wide topology: even-depth nodes, numbered by a scan
    uint32_t* flag = S.keys_b;  // free after the sort (unused by the SAH build)
    k_even_depth<<<grid_for(n_int, 256), 256, 0, s>>>(B, flag);
    k_scan_exclusive<<<1, 1024, 0, s>>>(flag, n_int);
    k_bin_to4<<<grid_for(n_int, 256), 256, 0, s>>>(B, flag);
    k_node4_topology<<<grid_for(n_int, 256), 256, 0, s>>>(B);
    k_validate<<<grid_for(n_int, 256), 256, 0, s>>>(B);
  }
  launch_refit(V, F, nf, bvh, scratch, s);
}

}  // namespace dt

// Traversal order of a depth level.  After the first bounce the rays of a
// level leave many surface points in many directions; a warp whose lanes
// carry unrelated rays spends most node visits with few lanes busy.  Rays
// that share a direction octant and leave nearby points take similar paths
// through the BVH, so every level k >= 1 can be traced in the order of a
// bucket key (ray_order_key: octant, then the Morton code of the origin; in
// a batch the scene index above them), and the traversal takes its
// segments bucket by bucket.  What is traced does not change: each
// segment's closest hit is written to its own record, so the results are
// the same in any order.
//
// A counting sort by bucket.  The shading pass of level k-1 writes each
// child's bucket and counts it in a table of 2^kOrderBits counters with an
// atomic whose return value is the child's rank in its bucket.  One scan turns the counts into bucket starts, and each segment's
// position in the order is then its bucket's start plus its rank: no sort
// passes.  The order within a bucket is the atomics' order; only the bucket
// sequence matters for coherence.  Keys and ranks live in the level's hit
// records (written only when the level is traced), the order in its flag
// words (written only by the shading pass after the trace), the table in a
// fixed region of the workspace.  Level sizes are read on the device, so
// the launches need no host synchronisation.
#include "dt_internal.cuh"

namespace dt {

constexpr int kOrderThreads = 256;
constexpr int kScanPerThread = 32;                           // counters per thread of the scan
constexpr int kScanSpan = kOrderThreads * kScanPerThread;    // counters per CTA of the scan

static_assert(kOrderCounters % kScanSpan == 0, "the counter table is a whole number of scan spans");
constexpr int kScanBlocks = kOrderCounters / kScanSpan;
static_assert(kScanBlocks <= 1024, "one CTA scans the span totals");

// Block-wide exclusive sum over kOrderThreads values; *total gets the sum.
__device__ __forceinline__ uint32_t block_exclusive_sum(uint32_t v, uint32_t* s_warp, uint32_t* total) {
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, x, o);
    if (lane >= (uint32_t)o) x += y;
  }
  if (lane == 31) s_warp[wid] = x;
  __syncthreads();
  uint32_t before = 0, all = 0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
    const uint32_t t = s_warp[w];
    if (w < (int)wid) before += t;
    all += t;
  }
  *total = all;
  return before + x - v;
}

// Counts -> exclusive starts within each span of kScanSpan counters; the
// span totals go to span_sum[].
__global__ void __launch_bounds__(kOrderThreads) k_order_scan_spans(uint32_t* __restrict__ count,
                                                                    uint32_t* __restrict__ span_sum) {
  __shared__ uint32_t s_warp[kOrderThreads / 32];
  uint4* c4 = reinterpret_cast<uint4*>(count + (size_t)blockIdx.x * kScanSpan + threadIdx.x * kScanPerThread);
  uint4 v[kScanPerThread / 4];
  uint32_t s = 0;
#pragma unroll
  for (int q = 0; q < kScanPerThread / 4; ++q) {
    v[q] = c4[q];
    s += v[q].x + v[q].y + v[q].z + v[q].w;
  }
  uint32_t total;
  uint32_t run = block_exclusive_sum(s, s_warp, &total);
#pragma unroll
  for (int q = 0; q < kScanPerThread / 4; ++q) {
    uint4 o;
    o.x = run; run += v[q].x;
    o.y = run; run += v[q].y;
    o.z = run; run += v[q].z;
    o.w = run; run += v[q].w;
    c4[q] = o;
  }
  if (threadIdx.x == 0) span_sum[blockIdx.x] = total;
}

// Exclusive scan of the span totals in place (one CTA).
__global__ void __launch_bounds__(1024) k_order_scan_totals(uint32_t* __restrict__ span_sum) {
  __shared__ uint32_t s_warp[32];
  const uint32_t v = threadIdx.x < (unsigned)kScanBlocks ? span_sum[threadIdx.x] : 0u;
  uint32_t total;
  const uint32_t e = block_exclusive_sum(v, s_warp, &total);
  if (threadIdx.x < (unsigned)kScanBlocks) span_sum[threadIdx.x] = e;
}

// Position of every segment of level k in the traversal order: its
// bucket's start plus its rank in the bucket.
__global__ void __launch_bounds__(kOrderThreads) k_order_place(WsView W, int k) {
  const WsHeader* H = W.hdr;
  const uint32_t n = level_size(H, k);
  const uint32_t start = H->level_start[k];
  const uint2* kr = level_buckets(W, k, start);
  uint32_t* order = W.sflag + start;
  const uint32_t* count = W.order_count;
  const uint32_t* span_sum = W.order_count + kOrderCounters;
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const uint2 br = kr[p];
    const uint32_t b = br.x & (kOrderCounters - 1);
    const uint32_t pos = __ldg(count + b) + __ldg(span_sum + b / kScanSpan) + br.y;
    if (pos < n) order[pos] = p;
  }
}

void launch_order_clear(const WsView& W, cudaStream_t s) {
  ProfScope ps("order_clear", s);
  cudaMemsetAsync(W.order_count, 0, (size_t)kOrderCounters * sizeof(uint32_t), s);
}

// Level k (k >= 1) into its traversal order, from the buckets and ranks the
// shading pass of level k-1 wrote.
void launch_order(const WsView& W, int k, cudaStream_t s) {
  ProfScope ps("k_order", s);
  uint32_t* span_sum = W.order_count + kOrderCounters;
  k_order_scan_spans<<<kScanBlocks, kOrderThreads, 0, s>>>(W.order_count, span_sum);
  k_order_scan_totals<<<1, 1024, 0, s>>>(span_sum);
  k_order_place<<<4 * num_sms(), kOrderThreads, 0, s>>>(W, k);
}

}  // namespace dt

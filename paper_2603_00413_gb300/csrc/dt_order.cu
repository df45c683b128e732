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
// child's bucket and counts it in a table of 2^kOrderBits counters.  One
// scan turns the counts into bucket starts, and a placement pass gives each
// segment the next free place of its bucket (an atomic on the start): no
// sort passes.  The order within a bucket is the atomics' order; only the
// bucket sequence matters for coherence.  The buckets live in the level's
// hit records (written only when the level is traced), the order in its
// flag words (written only by the shading pass after the trace), the table
// in a fixed region of the workspace.  Level sizes are read on the device,
// so the launches need no host synchronisation.
#include "dt_internal.cuh"

namespace dt {

constexpr int kOrderThreads = 256;
constexpr int kScanIters = 8;                                   // uint4 loads per lane
constexpr int kScanWarpSpan = kScanIters * 32 * 4;              // counters per warp of the scan
constexpr int kScanSpan = (kOrderThreads / 32) * kScanWarpSpan;  // counters per CTA of the scan (8192)

static_assert(kOrderCounters % kScanSpan == 0, "the counter table is a whole number of scan spans");
static_assert(kOrderCounters / kScanSpan <= 1024, "a CTA scans the span totals in shared memory");

// Inclusive warp sum of v over lanes 0..lane.
__device__ __forceinline__ uint32_t warp_inclusive_sum(uint32_t v) {
  const uint32_t lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, v, o);
    if (lane >= (uint32_t)o) v += y;
  }
  return v;
}

// Block-wide exclusive sum over the block's threads; *total gets the sum.
__device__ __forceinline__ uint32_t block_exclusive_sum(uint32_t v, uint32_t* s_warp, uint32_t* total) {
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint32_t x = warp_inclusive_sum(v);
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

// Counts -> exclusive starts within each span of kScanSpan counters (each
// warp an eighth of the span, read with coalesced 16-byte loads); the span
// totals go to span_sum[].
__global__ void __launch_bounds__(kOrderThreads) k_order_scan_spans(uint32_t* __restrict__ count,
                                                                    uint32_t* __restrict__ span_sum) {
  __shared__ uint32_t s_warp[kOrderThreads / 32];
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint4* c4 = reinterpret_cast<uint4*>(count + (size_t)blockIdx.x * kScanSpan + wid * kScanWarpSpan) + lane;
  uint4 v[kScanIters];
  uint32_t ex[kScanIters];
  uint32_t run = 0;  // the warp's sum so far
#pragma unroll
  for (int it = 0; it < kScanIters; ++it) v[it] = c4[it * 32];
#pragma unroll
  for (int it = 0; it < kScanIters; ++it) {
    const uint32_t s = v[it].x + v[it].y + v[it].z + v[it].w;
    const uint32_t inc = warp_inclusive_sum(s);
    ex[it] = run + inc - s;
    run += __shfl_sync(kFull, inc, 31);
  }
  uint32_t total;
  const uint32_t warp_base = block_exclusive_sum(lane == 0 ? run : 0u, s_warp, &total);
  const uint32_t base = __shfl_sync(kFull, warp_base, 0);
#pragma unroll
  for (int it = 0; it < kScanIters; ++it) {
    uint32_t r = base + ex[it];
    uint4 o;
    o.x = r; r += v[it].x;
    o.y = r; r += v[it].y;
    o.z = r; r += v[it].z;
    o.w = r;
    c4[it * 32] = o;
  }
  if (threadIdx.x == 0) span_sum[blockIdx.x] = total;
}

// Position of every segment of level k in the traversal order: the next
// free place of its bucket (an atomic on the bucket's start in its span,
// one per bucket per warp) plus the totals of the spans before it (scanned
// by each CTA in shared memory).  Four independent steps per warp keep
// several atomics in flight.
constexpr int kPlaceUnroll = 4;
__global__ void __launch_bounds__(kOrderThreads) k_order_place(WsView W, int k, int spans) {
  __shared__ uint32_t s_span[1024];
  __shared__ uint32_t s_warp[kOrderThreads / 32];
  const WsHeader* H = W.hdr;
  const uint32_t n = level_size(H, k);
  if (n == 0) return;
  const uint32_t start = H->level_start[k];
  {
    const uint32_t* tot = W.order_count + kOrderCounters;
    uint32_t v[4], sum = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = threadIdx.x * 4 + q;
      v[q] = j < spans ? tot[j] : 0u;
      sum += v[q];
    }
    uint32_t all;
    uint32_t run = block_exclusive_sum(sum, s_warp, &all);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      s_span[threadIdx.x * 4 + q] = run;
      run += v[q];
    }
  }
  __syncthreads();
  const uint32_t* kb = level_buckets(W, k, start);
  uint32_t* order = W.sflag + start;
  uint32_t* count = W.order_count;
  const uint32_t lane = threadIdx.x & 31;
  const unsigned lanes_below = (1u << lane) - 1u;
  const uint32_t stride = gridDim.x * blockDim.x;
  // warp-uniform loop: neighbouring segments often share a bucket, so the
  // lanes of one bucket take their places with one atomic
  for (uint32_t w0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); w0 < n; w0 += kPlaceUnroll * stride) {
    uint32_t b[kPlaceUnroll], base[kPlaceUnroll];
    unsigned peers[kPlaceUnroll];
#pragma unroll
    for (int j = 0; j < kPlaceUnroll; ++j) {
      const uint32_t p = w0 + j * stride + lane;
      b[j] = p < n ? kb[p] & (kOrderCounters - 1) : ~0u;
    }
#pragma unroll
    for (int j = 0; j < kPlaceUnroll; ++j) {
      peers[j] = __match_any_sync(kFull, b[j]);
      base[j] = 0;
      if (b[j] != ~0u && lane == (uint32_t)(__ffs(peers[j]) - 1))
        base[j] = atomicAdd(count + b[j], (uint32_t)__popc(peers[j]));
    }
#pragma unroll
    for (int j = 0; j < kPlaceUnroll; ++j) {
      const uint32_t c = __shfl_sync(kFull, base[j], __ffs(peers[j]) - 1) + __popc(peers[j] & lanes_below);
      if (b[j] == ~0u) continue;
      const uint32_t pos = c + s_span[b[j] / kScanSpan];
      if (pos < n) order[pos] = w0 + j * stride + lane;
    }
  }
}

// Buckets in use for `bits`-bit keys: whole scan spans.
static uint32_t order_buckets(int bits) {
  const uint32_t nb = 1u << bits;
  return nb < (uint32_t)kScanSpan ? (uint32_t)kScanSpan : nb;
}

void launch_order_clear(const WsView& W, int bits, cudaStream_t s) {
  ProfScope ps("order_clear", s);
  cudaMemsetAsync(W.order_count, 0, (size_t)order_buckets(bits) * sizeof(uint32_t), s);
}

// Level k (k >= 1) into its traversal order, from the buckets and ranks the
// shading pass of level k-1 wrote with `bits`-bit keys.
void launch_order(const WsView& W, int k, int bits, cudaStream_t s) {
  ProfScope ps("k_order", s);
  const int spans = (int)(order_buckets(bits) / kScanSpan);
  uint32_t* span_sum = W.order_count + kOrderCounters;
  k_order_scan_spans<<<spans, kOrderThreads, 0, s>>>(W.order_count, span_sum);
  k_order_place<<<8 * num_sms(), kOrderThreads, 0, s>>>(W, k, spans);
}

}  // namespace dt

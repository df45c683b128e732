// Traversal order of a depth level.  After the first bounce the rays of a
// level leave many surface points in many directions; a warp whose lanes
// carry unrelated rays spends most node visits with few lanes busy.  Rays
// that share a direction octant and leave nearby points take similar paths
// through the BVH, so every level k >= 1 is sorted by the key the shading
// pass of level k-1 writes with each segment (ray_order_key: octant, then
// the Morton code of the origin; in a batch the scene index above them) and
// the traversal takes its segments in that order.  What is traced does not
// change: each segment's closest hit is written to its own record, so the
// results are the same in any order.
//
// The sort is a stable LSD radix sort of 8-bit digits (3 passes for the
// 24-bit key, 4 with the scene index), each pass a histogram of contiguous
// per-CTA chunks, a scan per digit and a stable scatter.  It runs entirely
// in memory of level k that is free until the level is traced: the hit
// records (16 B per segment, four arrays of n 32-bit words A0..A3: the keys
// in A0, then temporaries) and the child and flag words (B0 = child,
// B1 = flag, written by the shading pass of level k after the trace).  The
// final order lands in B1, where k_trace reads it.  Level sizes are read on
// the device, so the launches need no host synchronisation.
#include "dt_internal.cuh"

namespace dt {

constexpr int kOrderThreads = 256;
constexpr int kOrderIpt = 8;                                // keys per thread per tile
constexpr int kOrderTile = kOrderThreads * kOrderIpt;       // 2048
constexpr int kOrderWarps = kOrderThreads / 32;

struct OrderIo {
  const uint32_t* kin;
  const uint32_t* vin;  // nullptr: the values are the positions (first pass)
  uint32_t* kout;       // nullptr: keys not kept (last pass)
  uint32_t* vout;
};

// Input and output arrays of pass `pass` of `npass` for level k of n segments.
__device__ __forceinline__ OrderIo order_io(const WsView& W, int k, uint32_t start, uint32_t n, int pass, int npass) {
  uint32_t* A = level_words(W, k, start);
  uint32_t* A1 = A + n;
  uint32_t* A2 = A + 2 * (size_t)n;
  uint32_t* A3 = A + 3 * (size_t)n;
  uint32_t* B0 = reinterpret_cast<uint32_t*>(W.child + start);
  uint32_t* B1 = W.sflag + start;
  if (pass == 0) return OrderIo{A, nullptr, A1, A2};
  if (pass == 1) return OrderIo{A1, A2, A3, B0};
  if (pass == npass - 1) return pass == 2 ? OrderIo{A3, B0, nullptr, B1} : OrderIo{A, A1, nullptr, B1};
  return OrderIo{A3, B0, A, A1};  // pass 2 of 4
}

// CTA b sorts positions [b c, (b + 1) c) of the level, c a multiple of the
// warp-group size
__device__ __forceinline__ uint32_t order_chunk(uint32_t n, uint32_t grid) {
  const uint32_t c = (n + grid - 1) / grid;
  return (c + kOrderThreads - 1) / kOrderThreads * kOrderThreads;
}

// Per-CTA digit counts of the CTA's chunk, digit-major: hist[d * grid + b].
__global__ void __launch_bounds__(kOrderThreads) k_order_hist(WsView W, int k, int pass, int npass) {
  const WsHeader* H = W.hdr;
  const uint32_t n = level_size(H, k);
  if (n == 0) return;
  const uint32_t start = H->level_start[k];
  const OrderIo io = order_io(W, k, start, n, pass, npass);
  const int shift = 8 * pass;
  const uint32_t lane = threadIdx.x & 31;
  __shared__ uint32_t cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const uint32_t c = order_chunk(n, gridDim.x);
  const uint32_t lo = min((uint32_t)blockIdx.x * c, n), hi = min(lo + c, n);
  for (uint32_t base = lo; base < hi; base += kOrderTile) {
    uint32_t dg[kOrderIpt];
#pragma unroll
    for (int j = 0; j < kOrderIpt; ++j) {
      const uint32_t i = base + j * kOrderThreads + threadIdx.x;
      dg[j] = i < hi ? (io.kin[i] >> shift) & 0xffu : 256u;
    }
#pragma unroll
    for (int j = 0; j < kOrderIpt; ++j) {
      // one shared atomic per distinct digit of the warp
      const unsigned peers = __match_any_sync(kFull, dg[j]);
      if (dg[j] < 256u && (uint32_t)(__ffs(peers) - 1) == lane) atomicAdd(&cnt[dg[j]], (uint32_t)__popc(peers));
    }
  }
  __syncthreads();
  W.order_hist[threadIdx.x * gridDim.x + blockIdx.x] = cnt[threadIdx.x];
}

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
  for (int w = 0; w < kOrderWarps; ++w) {
    const uint32_t t = s_warp[w];
    if (w < (int)wid) before += t;
    all += t;
  }
  *total = all;
  return before + x - v;
}

// Digit d (one CTA each): exclusive scan of its per-CTA counts in place, and
// the digit's total after the counts.
__global__ void __launch_bounds__(kOrderThreads) k_order_scan(WsView W, int k, int grid) {
  if (level_size(W.hdr, k) == 0) return;
  __shared__ uint32_t s_warp[kOrderWarps];
  uint32_t* h = W.order_hist + (size_t)blockIdx.x * grid;
  const int per = (grid + kOrderThreads - 1) / kOrderThreads;  // <= 4
  const int lo = threadIdx.x * per;
  uint32_t v[4] = {0u, 0u, 0u, 0u}, s = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (q < per && lo + q < grid) v[q] = h[lo + q];
    s += v[q];
  }
  uint32_t total;
  uint32_t run = block_exclusive_sum(s, s_warp, &total);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (q < per && lo + q < grid) {
      h[lo + q] = run;
      run += v[q];
    }
  }
  if (threadIdx.x == 0) W.order_hist[(size_t)256 * grid + blockIdx.x] = total;
}

// Stable scatter of each CTA's chunk: keys in chunk order, taken 256 at a
// time; the rank among equal digits comes from __match_any_sync within a
// warp and a per-step prefix over the warps' digit counts across warps.
__global__ void __launch_bounds__(kOrderThreads) k_order_scatter(WsView W, int k, int pass, int npass) {
  const WsHeader* H = W.hdr;
  const uint32_t n = level_size(H, k);
  if (n == 0) return;
  const uint32_t start = H->level_start[k];
  const OrderIo io = order_io(W, k, start, n, pass, npass);
  const int shift = 8 * pass;
  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t G = gridDim.x;
  __shared__ uint32_t s_warp[kOrderWarps];
  __shared__ uint32_t off[256];
  __shared__ uint32_t wcnt[kOrderWarps][256];
  __shared__ uint32_t wpre[kOrderWarps][256];
  {
    // where digit tid starts: the totals of the smaller digits plus this
    // CTA's scanned count
    uint32_t all;
    const uint32_t below = block_exclusive_sum(W.order_hist[(size_t)256 * G + tid], s_warp, &all);
    off[tid] = below + W.order_hist[(size_t)tid * G + blockIdx.x];
#pragma unroll
    for (int w = 0; w < kOrderWarps; ++w) wcnt[w][tid] = 0;
  }
  __syncthreads();
  const uint32_t c = order_chunk(n, G);
  const uint32_t lo = min((uint32_t)blockIdx.x * c, n), hi = min(lo + c, n);
  const unsigned lanes_below = (1u << lane) - 1u;
  uint32_t step_total = 0;  // digit tid's count in the previous step
  for (uint32_t base = lo; base < hi; base += kOrderTile) {
    uint32_t key[kOrderIpt], val[kOrderIpt];
#pragma unroll
    for (int j = 0; j < kOrderIpt; ++j) {
      const uint32_t i = base + j * kOrderThreads + tid;
      key[j] = 0u;
      val[j] = i;
      if (i < hi) {
        key[j] = io.kin[i];
        if (io.vin) val[j] = io.vin[i];
      }
    }
#pragma unroll
    for (int j = 0; j < kOrderIpt; ++j) {
      const uint32_t i = base + j * kOrderThreads + tid;
      const bool valid = i < hi;
      const uint32_t dg = valid ? (key[j] >> shift) & 0xffu : 256u;
      const unsigned peers = __match_any_sync(kFull, dg);
      const uint32_t rank = __popc(peers & lanes_below);
      if (valid && rank == 0) wcnt[warp][dg] = __popc(peers);
      __syncthreads();
      {
        // thread tid owns digit tid: advance past the previous step, then
        // the exclusive prefix over the warps of this step
        off[tid] += step_total;
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < kOrderWarps; ++w) {
          const uint32_t x = wcnt[w][tid];
          wcnt[w][tid] = 0;
          wpre[w][tid] = run;
          run += x;
        }
        step_total = run;
      }
      __syncthreads();
      if (valid) {
        const uint32_t pos = off[dg] + wpre[warp][dg] + rank;
        if (pos < n) {
          if (io.kout) io.kout[pos] = key[j];
          io.vout[pos] = val[j];
        }
      }
    }
  }
}

// Sorts level k (k >= 1) into its traversal order; npass 3 for one scene,
// 4 when the keys carry a scene index.
void launch_order(const WsView& W, int k, int npass, cudaStream_t s) {
  ProfScope ps("k_order", s);
  int grid = 4 * num_sms();
  if (grid > kOrderMaxBlocks) grid = kOrderMaxBlocks;
  for (int pass = 0; pass < npass; ++pass) {
    k_order_hist<<<grid, kOrderThreads, 0, s>>>(W, k, pass, npass);
    k_order_scan<<<256, kOrderThreads, 0, s>>>(W, k, grid);
    k_order_scatter<<<grid, kOrderThreads, 0, s>>>(W, k, pass, npass);
  }
}

}  // namespace dt

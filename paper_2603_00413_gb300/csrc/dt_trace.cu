// Forward wavefront of the recursive tracer (DiffTrans Sec. 3.4 "Recursive
// Ray Tracing", steps 1-5): camera rays into level 0, then per depth k a
// persistent closest-hit traversal of the LBVH and a shading pass that
// accumulates escaped rays into the image and appends the Fresnel-weighted
// reflected and refracted children to level k+1.
#include <cuda_runtime.h>
#include <stdint.h>

#include <string.h>

#include "dt_internal.cuh"
#include "dt_shade.cuh"
#include "dt_medium.cuh"

namespace dt {

// ---------------------------------------------------------------------------
// camera rays
// ---------------------------------------------------------------------------
__device__ __forceinline__ void jitter_offset(uint64_t seed, uint32_t view, uint32_t p, uint32_t s, float& jx,
                                              float& jy) {
  uint32_t h = pcg_hash((uint32_t)seed ^ pcg_hash((uint32_t)(seed >> 32)));
  h = pcg_hash(h ^ view);
  h = pcg_hash(h ^ p);
  h = pcg_hash(h ^ s);
  jx = (float)(pcg_hash(h) >> 8) * (1.0f / 16777216.0f);
  jy = (float)(pcg_hash(h ^ 0x9E3779B9u) >> 8) * (1.0f / 16777216.0f);
}

__device__ __forceinline__ void camera_ray(const float* cam, int width, int height, float sx, float sy, float3& o,
                                           float3& d) {
  const float3 eye = load3(cam), at = load3(cam + 3), up = load3(cam + 6);
  const float3 fwd = normalize(at - eye);
  float3 r = cross(fwd, up);
  if (len(r) < 1e-12f) r = cross(fwd, mk(0.f, 0.f, 1.f));
  r = normalize(r);
  const float3 u = cross(r, fwd);
  const float th = tanf(0.5f * cam[9] * kPi / 180.0f);
  const float aspect = (float)width / (float)height;
  const float px = (2.0f * sx / (float)width - 1.0f) * th * aspect;
  const float py = (1.0f - 2.0f * sy / (float)height) * th;
  o = eye;
  d = normalize(fwd + r * px + u * py);
}

// Scene table: the header and the entries arrive as kernel parameters (no
// host memcpy, so the writes are ordered on the stream and can be captured in
// a graph) and are copied into the workspace.
struct TableChunk {
  int32_t first, count;
  SceneEntry e[kEntriesPerChunk];
};
static_assert(sizeof(TableChunk) <= 32764, "a table chunk must fit the kernel-parameter space");

static_assert(sizeof(TableChunk) + sizeof(TableHeader) + 64 <= 32764,
              "the table header and a chunk must fit the kernel-parameter space together");

// One chunk of the table's entries, and with the first chunk the header.
__global__ void k_write_table(TableHeader* hdst, const TableHeader hsrc, SceneEntry* dst, const TableChunk src,
                              int with_header) {
  if (with_header) {
    const uint32_t* a = reinterpret_cast<const uint32_t*>(&hsrc);
    uint32_t* b = reinterpret_cast<uint32_t*>(hdst);
    for (int i = threadIdx.x; i < (int)(sizeof(TableHeader) / 4); i += blockDim.x) b[i] = a[i];
  }
  const int words = (int)(sizeof(SceneEntry) / 4);
  for (int i = threadIdx.x; i < src.count * words; i += blockDim.x) {
    const int k = i / words, w = i % words;
    reinterpret_cast<uint32_t*>(dst + src.first + k)[w] = reinterpret_cast<const uint32_t*>(&src.e[k])[w];
  }
}

// Pixel of position q of a view's pixels in traversal order: bands of four
// rows (the last one shorter when H is not a multiple of four), each taken
// column by column, so that 32 consecutive positions of a full band cover
// an 8x4 pixel block; a bijection of [0, W H).
__device__ __forceinline__ uint32_t tiled_pixel(uint32_t q, uint32_t w, uint32_t h) {
  const uint32_t band = q / (4u * w);
  const uint32_t hb = min(4u, h - 4u * band);
  const uint32_t r = q - band * 4u * w;
  return (4u * band + r % hb) * w + r / hb;
}

// Camera rays of every scene into level 0 (blockIdx.y = scene).  Sample
// index g = sample_start + (view * H * W + py * W + px) * spp + s; the
// samples of a view are laid out in the arena in tiled_pixel order (the
// samples of a pixel together), so that a warp's camera rays are an 8x4
// block of pixels rather than a row of 32.  The thread of a pixel's first
// sample also clears the pixel in the image the shading passes add to (one
// launch less per render than a clearing kernel of its own).
__global__ void k_camera(WsView W, unsigned long long capacity) {
  const SceneEntry& E = W.ent[blockIdx.y];
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
    W.hdr->capacity = capacity;
    W.hdr->ring = W.ring;
    W.hdr->mom = W.mom ? 1u : 0u;
    W.hdr->level_count[0] = W.th->n_samples;
    W.hdr->level_start[0] = 0;
  }
  const uint32_t npix = (uint32_t)E.width * (uint32_t)E.height;
  const uint32_t n0 = E.pix_count * (uint32_t)E.spp;
  for (uint32_t l = blockIdx.x * blockDim.x + threadIdx.x; l < n0; l += gridDim.x * blockDim.x) {
    const uint32_t s = l % (uint32_t)E.spp;
    const uint32_t gp = l / (uint32_t)E.spp;
    const uint32_t view = gp / npix;
    const uint32_t p = tiled_pixel(gp % npix, (uint32_t)E.width, (uint32_t)E.height);
    if (s == 0) {
      float* px = E.out + 3 * ((size_t)view * npix + p);
      px[0] = px[1] = px[2] = 0.0f;
    }
    float jx = 0.5f, jy = 0.5f;
    if (E.jitter) jitter_offset(E.seed, view, p, s, jx, jy);
    float3 o, d;
    camera_ray(E.cams + 10 * view, E.width, E.height, (float)(p % E.width) + jx, (float)(p / E.width) + jy, o, d);
    const uint32_t g = E.sample_start + (view * npix + p) * (uint32_t)E.spp + s;
    const uint32_t a = E.sample_start + l;
    W.ray_o[a] = make_float4(o.x, o.y, o.z, __uint_as_float(g));
    W.ray_d[a] = make_float4(d.x, d.y, d.z, __uint_as_float(1u));
    W.ray_w[a] = make_float4(1.f, 1.f, 1.f, __int_as_float(-1));
  }
}

// ---------------------------------------------------------------------------
// closest hit through the LBVH
// ---------------------------------------------------------------------------
// Slab test against one child box.  A zero direction component is replaced
// by +-1e-20 so no 0*inf NaN appears; the far distance is widened by
// 1 + 2*gamma(3) (Ize, "Robust BVH Ray Traversal", JCGT 2013) so rounding
// never culls a box the ray touches.
__device__ __forceinline__ bool slab(float3 o, float3 idir, float lox, float hix, float loy, float hiy, float loz,
                                     float hiz, float tmin, float tmax, float& tnear) {
  const float tx0 = (lox - o.x) * idir.x, tx1 = (hix - o.x) * idir.x;
  const float ty0 = (loy - o.y) * idir.y, ty1 = (hiy - o.y) * idir.y;
  const float tz0 = (loz - o.z) * idir.z, tz1 = (hiz - o.z) * idir.z;
  const float tn = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), tmin));
  const float tf = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fmaxf(tz0, tz1)) * 1.0000004f;
  tnear = tn;
  return tn <= fminf(tf, tmax);
}

__device__ __forceinline__ float safe_inv(float v) {
  return 1.0f / (fabsf(v) > 1e-20f ? v : copysignf(1e-20f, v));
}

struct ClosestHit {
  float t, b1, b2;
  int tri;
};

// Moller-Trumbore on a leaf; keeps the smallest t > tmin, ties to the smaller
// triangle id, skipping the triangle the ray starts on.
__device__ __forceinline__ void test_leaf(const float4* __restrict__ tris, int leaf, float3 o, float3 d, int src,
                                          float tmin, ClosestHit& h, uint32_t& ntest) {
  const float4 a = __ldg(tris + 3 * leaf), b = __ldg(tris + 3 * leaf + 1), c = __ldg(tris + 3 * leaf + 2);
  const int id = __float_as_int(a.w);
  if (id == src) return;
  ++ntest;
  // the arithmetic of intersect_known, written out (the checkpointed
  // backward calls that function on the same inputs and gets the same bits)
  const float3 v0 = xyz(a), e1 = xyz(b), e2 = xyz(c);
  const float3 p = cross(d, e2);
  const float det = dot(e1, p);
  if (det == 0.0f) return;
  const float inv = 1.0f / det;
  const float3 s = o - v0;
  const float b1 = dot(s, p) * inv;
  const float3 q = cross(s, e1);
  const float b2 = dot(d, q) * inv;
  const float t = dot(e2, q) * inv;
  const float b0 = 1.0f - b1 - b2;
  if (!(t > tmin)) return;
  if (b1 < 0.0f || b2 < 0.0f || b0 < 0.0f) return;
  if (t < h.t || (t == h.t && id < h.tri)) {
    h.t = t; h.b1 = b1; h.b2 = b2; h.tri = id;
  }
}

// Reads of BVH nodes with 256-bit loads (sm_100 and later): a 64-byte
// binary node is two loads instead of four 128-bit ones, which halves the
// load instructions a visit issues through L1 (the traversal is bound by
// instruction issue; measured 1.6 % faster than four 128-bit loads).  The
// BVH buffer is 256-byte aligned and every node starts at a multiple of 64
// bytes past it, so each load is 32-byte aligned.
__device__ __forceinline__ void ld_nc_v8(const float4* p, float4& a, float4& b) {
  asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
      : "l"(p));
}
__device__ __forceinline__ float4 ld_nc_l1na(const float4* p) {
  float4 r;
  asm("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];" : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w) : "l"(p));
  return r;
}
__device__ __forceinline__ void ld_node2(const float4* Np, float4& n0, float4& n1, float4& n2, int4& n3) {
  float4 c;
  ld_nc_v8(Np, n0, n1);
  ld_nc_v8(Np + 2, n2, c);
  n3 = make_int4(__float_as_int(c.x), __float_as_int(c.y), __float_as_int(c.z), __float_as_int(c.w));
}

// One visit of binary node `node`: slab tests on its two children, leaf
// children intersected at once, internal children that were hit entered
// nearest first with the other pushed.  Returns the next node, or -1 when the
// stack is empty.  (Used by the closest-hit tool; the persistent traversal
// uses visit_node2_deferred.)
__device__ __forceinline__ int visit_node2(const float4* __restrict__ node2, const float4* __restrict__ tris, int node,
                                           float3 o, float3 d, float3 idir, int src, float tmin, ClosestHit& h,
                                           int* stack, int& sp, bool& overflow, uint32_t& ntest) {
  float4 n0, n1, n2;
  int4 n3;
  ld_node2(node2 + 4 * node, n0, n1, n2, n3);
  float tn0, tn1;
  bool h0 = slab(o, idir, n0.x, n0.y, n0.z, n0.w, n2.x, n2.y, tmin, h.t, tn0);
  bool h1 = slab(o, idir, n1.x, n1.y, n1.z, n1.w, n2.z, n2.w, tmin, h.t, tn1);
  if (h0 && n3.x < 0) { test_leaf(tris, ~n3.x, o, d, src, tmin, h, ntest); h0 = false; }
  if (h1 && n3.y < 0) { test_leaf(tris, ~n3.y, o, d, src, tmin, h, ntest); h1 = false; }
  if (h0 && h1) {
    int nearc = n3.x, farc = n3.y;
    if (tn1 < tn0) { nearc = n3.y; farc = n3.x; }
    if (sp < kTraceStack) stack[sp++] = farc; else overflow = true;
    return nearc;
  }
  if (h0) return n3.x;
  if (h1) return n3.y;
  return sp > 0 ? stack[--sp] : -1;
}

// The binary visit of the persistent traversal: the same node test as
// visit_node2, but a hit leaf is queued in the lane's pending slots rather
// than intersected at once.  The kernel intersects every lane's pending
// triangles together after a few visits, so the triangle test runs as one
// block per few visits for the warp instead of one or two blocks per visit
// in which a few lanes work while the rest wait.  The caller visits only
// while fewer than two triangles are pending, so three slots always suffice.
__device__ __forceinline__ void push_pending(int leaf, int& p0, int& p1, int& p2) {
  if (p0 < 0) p0 = leaf;
  else if (p1 < 0) p1 = leaf;
  else p2 = leaf;
}
__device__ __forceinline__ int visit_node2_deferred(const float4* __restrict__ node2, int node, float3 o, float3 idir,
                                                    float tmin, float tmax, int* stack, int& sp, bool& overflow,
                                                    int& p0, int& p1, int& p2) {
  float4 n0, n1, n2;
  int4 n3;
  ld_node2(node2 + 4 * node, n0, n1, n2, n3);
  float tn0, tn1;
  bool h0 = slab(o, idir, n0.x, n0.y, n0.z, n0.w, n2.x, n2.y, tmin, tmax, tn0);
  bool h1 = slab(o, idir, n1.x, n1.y, n1.z, n1.w, n2.z, n2.w, tmin, tmax, tn1);
  if (h0 && n3.x < 0) { push_pending(~n3.x, p0, p1, p2); h0 = false; }
  if (h1 && n3.y < 0) { push_pending(~n3.y, p0, p1, p2); h1 = false; }
  if (h0 && h1) {
    int nearc = n3.x, farc = n3.y;
    if (tn1 < tn0) { nearc = n3.y; farc = n3.x; }
    if (sp < kTraceStack) stack[sp++] = farc; else overflow = true;
    return nearc;
  }
  if (h0) return n3.x;
  if (h1) return n3.y;
  return sp > 0 ? stack[--sp] : -1;
}

// The 4-wide visit of the persistent traversal, with hit leaves queued as
// in visit_node2_deferred (the caller visits only while nothing is pending,
// so four slots suffice).
__device__ __forceinline__ void push_pending4(int leaf, int& p0, int& p1, int& p2, int& p3) {
  if (p0 < 0) p0 = leaf;
  else if (p1 < 0) p1 = leaf;
  else if (p2 < 0) p2 = leaf;
  else p3 = leaf;
}
__device__ __forceinline__ int visit_node4_deferred(const float4* __restrict__ node4, int node, float3 o, float3 idir,
                                                    float tmin, float tmax, int* stack, int& sp, bool& overflow,
                                                    int& p0, int& p1, int& p2, int& p3) {
  const float4* Np = node4 + 8 * node;
  float4 lx, hx, ly, hy, lz, hz, chf, pad;
  ld_nc_v8(Np, lx, hx);
  ld_nc_v8(Np + 2, ly, hy);
  ld_nc_v8(Np + 4, lz, hz);
  ld_nc_v8(Np + 6, chf, pad);
  const int4 ch = make_int4(__float_as_int(chf.x), __float_as_int(chf.y), __float_as_int(chf.z), __float_as_int(chf.w));
  float t0, t1, t2, t3;
  bool b0 = ch.x != kNoChild && slab(o, idir, lx.x, hx.x, ly.x, hy.x, lz.x, hz.x, tmin, tmax, t0);
  bool b1 = ch.y != kNoChild && slab(o, idir, lx.y, hx.y, ly.y, hy.y, lz.y, hz.y, tmin, tmax, t1);
  bool b2 = ch.z != kNoChild && slab(o, idir, lx.z, hx.z, ly.z, hy.z, lz.z, hz.z, tmin, tmax, t2);
  bool b3 = ch.w != kNoChild && slab(o, idir, lx.w, hx.w, ly.w, hy.w, lz.w, hz.w, tmin, tmax, t3);
  if (b0 && ch.x < 0) { push_pending4(~ch.x, p0, p1, p2, p3); b0 = false; }
  if (b1 && ch.y < 0) { push_pending4(~ch.y, p0, p1, p2, p3); b1 = false; }
  if (b2 && ch.z < 0) { push_pending4(~ch.z, p0, p1, p2, p3); b2 = false; }
  if (b3 && ch.w < 0) { push_pending4(~ch.w, p0, p1, p2, p3); b3 = false; }
  float ta = b0 ? t0 : INFINITY, tb = b1 ? t1 : INFINITY, tc = b2 ? t2 : INFINITY, td = b3 ? t3 : INFINITY;
  int ra = ch.x, rb = ch.y, rc = ch.z, rd = ch.w;
  const int cnt = b0 + b1 + b2 + b3;
  if (cnt == 0) return sp > 0 ? stack[--sp] : -1;
#define DT_CSWAP(ta_, ra_, tb_, rb_)                     \
  if (tb_ < ta_) {                                      \
    const float tt = ta_; ta_ = tb_; tb_ = tt;          \
    const int rr = ra_; ra_ = rb_; rb_ = rr;            \
  }
  DT_CSWAP(ta, ra, tb, rb) DT_CSWAP(tc, rc, td, rd) DT_CSWAP(ta, ra, tc, rc) DT_CSWAP(tb, rb, td, rd)
  DT_CSWAP(tb, rb, tc, rc)
#undef DT_CSWAP
  if (sp + cnt - 1 > kTraceStack) {
    overflow = true;
    return ra;
  }
  if (cnt >= 4) stack[sp++] = rd;
  if (cnt >= 3) stack[sp++] = rc;
  if (cnt >= 2) stack[sp++] = rb;
  return ra;
}


// A tree traversal visits every node at most once, so more than max_iter
// = 2 n_int + 8 visits means a corrupt hierarchy: give up and flag it.
__device__ __forceinline__ ClosestHit closest_hit(const float4* __restrict__ node2, const float4* __restrict__ tris,
                                                  float3 o, float3 d, int src, float tmin, int max_iter,
                                                  uint32_t& nvis, uint32_t& ntest, bool& overflow) {
  ClosestHit h{INFINITY, 0.f, 0.f, -1};
  const float3 idir = mk(safe_inv(d.x), safe_inv(d.y), safe_inv(d.z));
  int stack[kTraceStack];
  int sp = 0;
  int node = 0;
  for (int it = 0; node >= 0; ++it) {
    if (it >= max_iter) {
      overflow = true;
      break;
    }
    ++nvis;
    node = visit_node2(node2, tris, node, o, d, idir, src, tmin, h, stack, sp, overflow, ntest);
  }
  return h;
}

// Persistent traversal of level k with dynamic refill.  Every lane carries
// its own ray; a warp runs up to `steps` node visits per round, then, when
// at least `refill` lanes have finished, hands them new segments from a
// batch of kTraceClaim it claimed from the level's cursor with one atomic.
// Within a round, leaves hit by a visit are queued per lane and intersected
// for the whole warp every kLeafEvery visits.  A warp stops when the level
// is exhausted and its last ray is done.  sorted != 0: position i of the
// level is the segment the traversal order put there (its flag word holds
// it until the shading pass rewrites it).
// kBatch = false: one scene, whose entry E0 arrives as a kernel parameter
// (uniform constant-bank reads); true: each ray looks its scene up.
constexpr int kTraceClaim = 64;  // segments a warp claims from the level cursor at once
constexpr int kLeafEvery = 6;    // node visits between the warp's batched triangle tests

template <int kMinBlocks, int kWidth, bool kBatch>
__global__ void __launch_bounds__(256, kMinBlocks) k_trace(WsView W, int k, int steps, int refill,
                                                           const SceneEntry E0, int sorted) {
  WsHeader* H = W.hdr;
  uint32_t* cursor = &H->fetch[k];
  const int n_scenes = kBatch ? W.th->n : 1;
  const uint32_t n = level_size(H, k);
  const uint32_t start = H->level_start[k];
  // the level's traversal order (dt_order.cu), or its arena order
  const uint32_t* order = sorted ? W.sflag + start : nullptr;
  const uint32_t lane = threadIdx.x & 31;
  const unsigned lanes_below = (1u << lane) - 1u;
  uint32_t nvis = 0, ntest = 0;
  bool overflow = false;
  bool active = false, exhausted = false;
  uint32_t a = 0;
  float3 o = mk(0.f, 0.f, 0.f), d = o, idir = o;
  int src = -1, node = 0, sp = 0, iters = 0;
  int max_iter = kBatch ? 0 : (E0.bh->corrupt ? 0 : E0.max_iter);  // a tree that failed validation is not traced
  float tmin = E0.t_min;
  const float4* nodes = kWidth == 4 ? E0.node4 : E0.node2;
  const float4* tris = E0.tris;
  ClosestHit h{INFINITY, 0.f, 0.f, -1};
  int stack[kTraceStack];
  // the warp's claimed batch [qb, qe) of the level's segments: one atomic on
  // the level cursor per kTraceClaim segments, not one per refill.  Warp w
  // starts with batch w of the level without an atomic, of B =
  // min(kTraceClaim, max(4, ceil(n / warps))) segments; the cursor hands out the
  // batches after the first of every warp.  A level smaller than
  // kTraceClaim segments per warp is thus spread over every warp (a few
  // thousand segments, as in a 64x64 frame, would otherwise sit in a few
  // dozen warps whose rays run one after another), and a warp past its end
  // leaves at once instead of queueing an atomic on the one cursor address.
  const uint32_t warps = gridDim.x * blockDim.x / 32u;
  uint32_t first = (n + warps - 1u) / warps;
  if (first < 4u) first = 4u;  // at least 4 rays a warp: one ray a warp leaves issue slots to idle lanes
  if (first > (uint32_t)kTraceClaim) first = kTraceClaim;
  const uint32_t static_span = warps * first;
  uint32_t qb = ((blockIdx.x * blockDim.x + threadIdx.x) / 32u) * first, qe = qb + first;
  if (qb > n) qb = n;
  if (qe > n) qe = n;
  bool cursor_done = static_span >= n;
  while (true) {
    const unsigned idle = __ballot_sync(kFull, !active);
    const int n_idle = __popc(idle);
    if (!exhausted && n_idle >= refill) {
      const uint32_t have = qe - qb;
      uint32_t nb = 0;
      const bool claim = have < (uint32_t)n_idle && !cursor_done;
      if (claim) {
        if (lane == 0) nb = atomicAdd(cursor, (uint32_t)kTraceClaim) + static_span;
        nb = __shfl_sync(kFull, nb, 0);
      }
      const uint32_t r = __popc(idle & lanes_below);
      const uint32_t i = r < have ? qb + r : (claim ? nb + (r - have) : 0xffffffffu);
      if (claim) {
        const uint32_t used = (uint32_t)n_idle - have;
        qb = nb + used;
        qe = nb + (uint32_t)kTraceClaim;
        if (nb + (uint32_t)kTraceClaim >= n) cursor_done = true;
      } else {
        qb += min((uint32_t)n_idle, have);
      }
      if (qe > n) qe = n;
      if (qb > qe) qb = qe;
      if (cursor_done && qb >= qe) exhausted = true;
      if (!active && i < n) {
        const uint32_t pos = order ? __ldg(order + i) : i;
        if (pos >= n) overflow = true;  // not a permutation of the level: reported, not traced
        else {
          a = start + pos;
          // read once here: not allocated in L1, so they do not evict BVH
          // nodes (L2 keeps them for the shading pass that follows)
          const float4 ro = ld_nc_l1na(W.ray_o + a), rd = ld_nc_l1na(W.ray_d + a), rw = ld_nc_l1na(W.ray_w + a);
          if (kBatch) {
            const SceneEntry& E = W.ent[find_scene(W.th->starts, n_scenes, __float_as_uint(ro.w))];
            nodes = kWidth == 4 ? E.node4 : E.node2;
            tris = E.tris;
            max_iter = E.bh->corrupt ? 0 : E.max_iter;
            tmin = E.t_min;
          }
          o = xyz(ro);
          d = xyz(rd);
          idir = mk(safe_inv(d.x), safe_inv(d.y), safe_inv(d.z));
          src = __float_as_int(rw.w);
          h = ClosestHit{INFINITY, 0.f, 0.f, -1};
          node = 0;
          sp = 0;
          iters = 0;
          active = true;
        }
      }
    }
    if (!__any_sync(kFull, active)) break;
    if (!active) continue;
    // A valid tree is visited at most once per node (max_iter = 2 n_int + 8);
    // the guard is checked once per round, so a corrupt tree (max_iter 0) is
    // never entered and a runaway ray stops within one round of the bound.
    int st = 0;
    bool done = iters >= max_iter;
    if (!done) {
      if (kWidth == 2) {
        // visits in groups of kLeafEvery, then the pending triangles of the
        // whole warp at once (see visit_node2_deferred)
        int p0 = -1, p1 = -1, p2 = -1;
        while (st < steps) {
          for (int j = 0; j < kLeafEvery && node >= 0 && p1 < 0; ++j, ++st)
            node = visit_node2_deferred(nodes, node, o, idir, tmin, h.t, stack, sp, overflow, p0, p1, p2);
          if (p0 >= 0) test_leaf(tris, p0, o, d, src, tmin, h, ntest);
          if (p1 >= 0) test_leaf(tris, p1, o, d, src, tmin, h, ntest);
          if (p2 >= 0) test_leaf(tris, p2, o, d, src, tmin, h, ntest);
          p0 = p1 = p2 = -1;
          if (node < 0) {
            done = true;
            break;
          }
        }
      } else {
        int p0 = -1, p1 = -1, p2 = -1, p3 = -1;
        while (st < steps) {
          for (int j = 0; j < kLeafEvery && node >= 0 && p0 < 0; ++j, ++st)
            node = visit_node4_deferred(nodes, node, o, idir, tmin, h.t, stack, sp, overflow, p0, p1, p2, p3);
          if (p0 >= 0) test_leaf(tris, p0, o, d, src, tmin, h, ntest);
          if (p1 >= 0) test_leaf(tris, p1, o, d, src, tmin, h, ntest);
          if (p2 >= 0) test_leaf(tris, p2, o, d, src, tmin, h, ntest);
          if (p3 >= 0) test_leaf(tris, p3, o, d, src, tmin, h, ntest);
          p0 = p1 = p2 = p3 = -1;
          if (node < 0) {
            done = true;
            break;
          }
        }
      }
      nvis += (uint32_t)st;
      iters += st;
      if (!done && iters >= max_iter) done = true;
    }
    if (done) {
      if (node >= 0) overflow = true;  // stopped by the guard
      W.hit[hit_slot(W, k, a, a - start)] = h.tri >= 0 ? make_float4(h.t, h.b1, h.b2, __int_as_float(h.tri))
                                                       : make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
      active = false;
    }
  }
  // the visit and test counts, summed over the CTA first: with a small level
  // spread over every warp, one atomic per warp on these two addresses would
  // queue thousands of atomics at the end of the launch
  __shared__ unsigned long long s_count[2];
  if (threadIdx.x == 0) s_count[0] = s_count[1] = 0ull;
  __syncthreads();
  const unsigned wv = __reduce_add_sync(kFull, nvis), wt = __reduce_add_sync(kFull, ntest);
  if (lane == 0) {
    if (wv) atomicAdd(&s_count[0], (unsigned long long)wv);
    if (wt) atomicAdd(&s_count[1], (unsigned long long)wt);
  }
  if (__any_sync(kFull, overflow) && lane == 0) atomicOr(&H->status, ST_STACK_OVERFLOW);
  __syncthreads();
  if (threadIdx.x == 0 && s_count[0]) atomicAdd(&H->counters[CNT_NODES], s_count[0]);
  if (threadIdx.x == 1 && s_count[1]) atomicAdd(&H->counters[CNT_TRIS], s_count[1]);
}

// Closest hit of arbitrary rays (tooling and tests).
__global__ void k_closest_hit_rays(const float4* __restrict__ nodes, const float4* __restrict__ tris,
                                   const float* __restrict__ o, const float* __restrict__ d,
                                   const int32_t* __restrict__ src, int32_t n, const BvhHeader* bh, float tmin,
                                   int max_iter, int32_t* __restrict__ tri, float* __restrict__ tbb) {
  const bool corrupt = bh->corrupt != 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    uint32_t nv = 0, nt = 0;
    bool ovf = false;
    if (corrupt) {
      tri[i] = -2;
      continue;
    }
    const ClosestHit h = closest_hit(nodes, tris, load3(o + 3 * i), load3(d + 3 * i), src ? src[i] : -1, tmin,
                                     max_iter, nv, nt, ovf);
    tri[i] = ovf ? -2 : h.tri;
    tbb[3 * i] = h.tri >= 0 ? h.t : 0.f;
    tbb[3 * i + 1] = h.b1;
    tbb[3 * i + 2] = h.b2;
  }
}

// ---------------------------------------------------------------------------
// shading: Sec. 3.4 steps 1-5 for every segment of level k
// ---------------------------------------------------------------------------
// Shading of every segment of level k: Sec. 3.4 steps 1-5 with the
// segment's own scene (depth limit, materials, environment, image); kBatch
// as for k_trace.
constexpr int kShadeThreads = 256;
constexpr int kShadeMinBlocks = 4;  // CTAs per SM the register budget is sized for

// order_bits != 0: each child is also counted in its traversal-order
// bucket (order_bucket of ray_order_key with that many bits; dt_order.cu)
// and its bucket is stored with the next level.  kGrid: 1 = some scene has
// an absorption grid, whose optical depth interior segments add
// (dt_medium.cuh); 2 = some scene's is a hash texture.
template <bool kBatch, int kGrid>
__global__ void __launch_bounds__(kShadeThreads, kShadeMinBlocks) k_shade(WsView W, int k, const SceneEntry E0,
                                                                         int order_bits) {
  WsHeader* H = W.hdr;
  const int n_scenes = kBatch ? W.th->n : 1;
  const uint32_t n = level_size(H, k);
  const uint32_t start = H->level_start[k];
  const uint32_t next_start = start + n;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    H->level_start[k + 1] = next_start;
    if (n) H->n_levels = (uint32_t)(k + 1);
  }
  __shared__ uint32_t s_wr[kShadeThreads / 32], s_wt[kShadeThreads / 32];
  __shared__ uint32_t s_base, s_nr;
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t* next_kr = order_bits ? level_buckets(W, k + 1, next_start) : nullptr;
  // positions of level k+1 that can hold a bucket (its ring half, or the arena)
  const unsigned long long key_room = W.ring ? (unsigned long long)W.ring : H->capacity - next_start;
  float3 box_lo = mk(0.f, 0.f, 0.f), box_scale = box_lo;
  if (!kBatch && order_bits) scene_order_box(E0.node2, box_lo, box_scale);
  uint32_t c_hit = 0, c_miss = 0, c_disc = 0, c_back = 0, c_tir = 0, c_med = 0;
  bool overflow = false;
  // CTA-wide tiles, so that the children of a tile are appended with one
  // atomic on the level counter per CTA rather than per warp
  for (uint32_t tile = blockIdx.x * kShadeThreads; tile < n; tile += gridDim.x * kShadeThreads) {
    const uint32_t i = tile + threadIdx.x;
    const uint32_t a = start + i;
    int nchild = 0;
    uint32_t fl = 0, scene_id = 0;
    uint32_t b_r = ~0u, p_r = 0, b_t = ~0u, p_t = 0;  // order buckets and next-level positions of the children
    float4 co = make_float4(0.f, 0.f, 0.f, 0.f), cdr = co, cwr = co, cdt = co, cwt = co;
    if (i < n) {
      const float4 ro = W.ray_o[a], rd = W.ray_d[a], rw = W.ray_w[a], hh = W.hit[hit_slot(W, k, a, i)];
      const uint32_t sample = __float_as_uint(ro.w);
      const int scene = kBatch ? find_scene(W.th->starts, n_scenes, sample) : 0;
      const SceneEntry& E = kBatch ? W.ent[scene] : E0;
      const int tri = __float_as_int(hh.w);
      const float3 d = xyz(rd);
      if (tri < 0) {  // step 3: no intersection -> environment
        fl = SF_MISS;
        ++c_miss;
        const uint32_t pix = (sample - E.sample_start) / (uint32_t)E.spp;
        if (sample >= E.sample_start && pix < E.pix_count) {  // dead records carry an out-of-range sample
          const float3 Ev = env_lookup(E.env, E.env_w, E.env_h, d);
          const float inv_spp = 1.0f / (float)E.spp;
          float* dst = E.out + 3 * (size_t)pix;
          atomicAdd(dst + 0, rw.x * Ev.x * inv_spp);
          atomicAdd(dst + 1, rw.y * Ev.y * inv_spp);
          atomicAdd(dst + 2, rw.z * Ev.z * inv_spp);
        }
      } else {
        ++c_hit;
        const int i0 = __ldg(E.F + 3 * tri), i1 = __ldg(E.F + 3 * tri + 1), i2 = __ldg(E.F + 3 * tri + 2);
        const float3 v0 = load3(E.V + 3 * i0), v1 = load3(E.V + 3 * i1), v2 = load3(E.V + 3 * i2);
        if (k >= E.max_depth) {  // step 1: the depth limit: contributes nothing
          const float3 ng = cross(v1 - v0, v2 - v0);
          fl = SF_DISCARDED | (dot(d, ng) < 0.0f ? 0u : SF_INSIDE);
          ++c_disc;
        } else {
          const float ior = __ldg(E.ior);
          const float3 sigma = mk(__ldg(E.sigma), __ldg(E.sigma + 1), __ldg(E.sigma + 2));
          HitShade h;
          shade_hit(xyz(ro), d, hh.x, hh.y, hh.z, v0, v1, v2, load3(E.N + 3 * i0), load3(E.N + 3 * i1),
                    load3(E.N + 3 * i2), ior, sigma, h);
          if (kGrid && E.mu && !h.entering) {  // Sec. 3.4 step 5 with the grid's optical depth
            // tape_mode 2: the medium pass has marched it (S_0 = NaN: not marched there)
            float3 S = mk(NAN, 0.f, 0.f);
            if (W.mom) S = mk(W.mom[(kMomS + 0) * W.cap + a], W.mom[(kMomS + 1) * W.cap + a], W.mom[(kMomS + 2) * W.cap + a]);
            if (isnan(S.x)) {
              S = medium_depth<kGrid == 2>(medium_view(E, W.ent + scene), xyz(ro), d, hh.x);
              c_med += (uint32_t)medium_full_steps(hh.x, E.gstep) + 1u;
            }
            h.A = absorption_with_depth(sigma, hh.x, S);
          }
          fl = h.entering ? 0u : SF_INSIDE;
          if (h.backfacing) {
            fl |= SF_BACKFACING;
            ++c_back;
          } else {
            if (h.tir) { fl |= SF_TIR; ++c_tir; }
            const uint32_t node = __float_as_uint(rd.w);
            const float3 Wt = mk(rw.x * h.A.x, rw.y * h.A.y, rw.z * h.A.z);
            co = make_float4(h.x.x, h.x.y, h.x.z, ro.w);
            cdr = make_float4(h.wr.x, h.wr.y, h.wr.z, __uint_as_float(2u * node));
            cwr = make_float4(Wt.x * h.R, Wt.y * h.R, Wt.z * h.R, __int_as_float(tri));
            nchild = 1;
            if (kBatch && order_bits) {
              scene_order_box(E.node2, box_lo, box_scale);
              scene_id = (uint32_t)scene;
            }
            if (!h.tir) {
              cdt = make_float4(h.wt.x, h.wt.y, h.wt.z, __uint_as_float(2u * node + 1u));
              cwt = make_float4(Wt.x * h.T, Wt.y * h.T, Wt.z * h.T, __int_as_float(tri));
              nchild = 2;
            }
          }
        }
      }
    }
    // CTA-aggregated append of the children to level k+1, the tile's
    // reflected children first and its refracted ones after them: rays of
    // one kind from neighbouring parents take similar paths, so the next
    // level's warps diverge less than with the two kinds interleaved.  Warp
    // ballots, a prefix over the warps, one atomic per tile.
    const unsigned br = __ballot_sync(kFull, nchild > 0), bt = __ballot_sync(kFull, nchild == 2);
    if (lane == 0) {
      s_wr[wid] = __popc(br);
      s_wt[wid] = __popc(bt);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t rr = 0, tt = 0;
      for (int w = 0; w < kShadeThreads / 32; ++w) {
        const uint32_t x = s_wr[w], y = s_wt[w];
        s_wr[w] = rr;
        s_wt[w] = tt;
        rr += x;
        tt += y;
      }
      s_base = (rr + tt) ? atomicAdd(&H->level_count[k + 1], rr + tt) : 0u;
      s_nr = rr;
    }
    __syncthreads();
    const uint32_t tile_base = s_base, tile_nr = s_nr, off_r = s_wr[wid], off_t = s_wt[wid];
    __syncthreads();  // the shared offsets are rewritten by the next tile
    if (i < n) {
      int32_t ch = -1;
      uint32_t delta = 0;
      if (nchild > 0) {
        // every allocated position below the capacity is written by exactly
        // one child; a child past the capacity is dropped (overflow)
        const uint32_t below = (1u << lane) - 1u;
        const unsigned long long jr = (unsigned long long)next_start + tile_base + off_r + __popc(br & below);
        if (jr < H->capacity) {
          ch = (int32_t)jr;
          W.ray_o[jr] = co; W.ray_d[jr] = cdr; W.ray_w[jr] = cwr;
          if (next_kr && jr - next_start < key_room) {
            p_r = (uint32_t)(jr - next_start);
            b_r = order_bucket(ray_order_key(xyz(co), xyz(cdr), box_lo, box_scale), order_bits, kBatch, scene_id);
          }
        } else {
          overflow = true;
        }
        if (nchild == 2) {
          const unsigned long long jt =
              (unsigned long long)next_start + tile_base + tile_nr + off_t + __popc(bt & below);
          delta = (uint32_t)(jt - jr);
          if (jt < H->capacity) {
            W.ray_o[jt] = co; W.ray_d[jt] = cdt; W.ray_w[jt] = cwt;
            if (next_kr && jt - next_start < key_room) {
              p_t = (uint32_t)(jt - next_start);
              b_t = order_bucket(ray_order_key(xyz(co), xyz(cdt), box_lo, box_scale), order_bits, kBatch, scene_id);
            }
          } else {
            overflow = true;
          }
        }
      }
      W.child[a] = ch;
      W.sflag[a] = fl | (delta << kRefractShift);
    }
    if (next_kr) {
      order_count_child(W.order_count, next_kr, b_r, p_r);
      order_count_child(W.order_count, next_kr, b_t, p_t);
    }
  }
  warp_add_u64(&H->counters[CNT_HITS], c_hit);
  warp_add_u64(&H->counters[CNT_MISSES], c_miss);
  warp_add_u64(&H->counters[CNT_DISCARDED], c_disc);
  warp_add_u64(&H->counters[CNT_BACKFACING], c_back);
  warp_add_u64(&H->counters[CNT_TIR], c_tir);
  if (kGrid) warp_add_u64(&H->counters[CNT_MEDIUM], c_med);
  if (__any_sync(kFull, overflow) && lane == 0) atomicOr(&H->status, ST_QUEUE_OVERFLOW);
}

// The medium pass of tape_mode 2, between the traversal and the shading of
// level k: for every segment that hits from inside (the shading pass's test
// of the geometric normal) in a scene with an absorption grid or hash
// texture, the optical depth over the segment and its derivatives
// (medium_moments) into the moments arrays; a segment found entering gets
// S_0 = NaN, so a shading pass that rounds the test the other way marches
// it itself.  A pass of its own: the march's accumulators need more
// registers than the shading pass runs with.  A warp classifies 32
// positions at a time (hit, a medium, not at the depth limit, from inside),
// queues the interior ones in shared memory and marches them 32 at a time,
// so its lanes march together rather than beside lanes whose segment needs
// no march.
constexpr int kMedFwdWarps = 8;
template <bool kBatch, bool kHash>
__global__ void __launch_bounds__(32 * kMedFwdWarps, 2) k_medium_forward(WsView W, int k, const SceneEntry E0) {
  __shared__ uint32_t s_queue[kMedFwdWarps][64];
  WsHeader* H = W.hdr;
  const int n_scenes = kBatch ? W.th->n : 1;
  const uint32_t n = level_size(H, k);
  const uint32_t start = H->level_start[k];
  const unsigned long long cap = W.cap;
  float* __restrict__ M = W.mom;
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t* q = s_queue[wid];
  const uint32_t warps = gridDim.x * kMedFwdWarps;
  uint32_t c_med = 0, cnt = 0;
  for (uint32_t base = (blockIdx.x * kMedFwdWarps + wid) * 32u;; base += warps * 32u) {
    const bool more = base < n;
    if (more) {
      const uint32_t i = base + lane;
      bool v = false;
      if (i < n) {
        const uint32_t a = start + i;
        const float4 hh = W.hit[hit_slot(W, k, a, i)];
        const int tri = __float_as_int(hh.w);
        if (tri >= 0) {
          const float4 rd = W.ray_d[a];
          const int scene = kBatch ? find_scene(W.th->starts, n_scenes, __float_as_uint(W.ray_o[a].w)) : 0;
          const SceneEntry& E = kBatch ? W.ent[scene] : E0;
          if (E.mu && k < E.max_depth) {
            const int i0 = __ldg(E.F + 3 * tri), i1 = __ldg(E.F + 3 * tri + 1), i2 = __ldg(E.F + 3 * tri + 2);
            const float3 v0 = load3(E.V + 3 * i0), v1 = load3(E.V + 3 * i1), v2 = load3(E.V + 3 * i2);
            if (dot(xyz(rd), cross(v1 - v0, v2 - v0)) < 0.0f) M[kMomS * cap + a] = NAN;  // entering: no medium
            else v = true;
          }
        }
      }
      const unsigned b = __ballot_sync(kFull, v);
      if (v) q[cnt + __popc(b & ((1u << lane) - 1u))] = i;
      cnt += (uint32_t)__popc(b);
      __syncwarp();
    }
    while (cnt >= 32u || (!more && cnt > 0u)) {
      const uint32_t take = cnt < 32u ? cnt : 32u;
      if (lane < take) {
        const uint32_t i = q[lane], a = start + i;
        const float4 hh = W.hit[hit_slot(W, k, a, i)];
        const float4 ro = W.ray_o[a], rd = W.ray_d[a];
        const int scene = kBatch ? find_scene(W.th->starts, n_scenes, __float_as_uint(ro.w)) : 0;
        const SceneEntry& E = kBatch ? W.ent[scene] : E0;
        const MediumMoments m = medium_moments<kHash>(medium_view(E, W.ent + scene), xyz(ro), xyz(rd), hh.x);
        c_med += (uint32_t)medium_full_steps(hh.x, E.gstep) + 1u;
        const float v[kMomFloats] = {m.S.x,  m.S.y,  m.S.z,  m.dt.x, m.dt.y, m.dt.z, m.ox.x, m.oy.x,
                                     m.oz.x, m.ox.y, m.oy.y, m.oz.y, m.ox.z, m.oy.z, m.oz.z, m.dx.x,
                                     m.dy.x, m.dz.x, m.dx.y, m.dy.y, m.dz.y, m.dx.z, m.dy.z, m.dz.z};
#pragma unroll
        for (int j = 0; j < kMomFloats; ++j) M[j * cap + a] = v[j];
      }
      __syncwarp();
      const uint32_t rest = cnt - take;
      const uint32_t x = lane < rest ? q[take + lane] : 0u;
      __syncwarp();
      if (lane < rest) q[lane] = x;
      __syncwarp();
      cnt = rest;
    }
    if (!more) break;
  }
  warp_add_u64(&H->counters[CNT_MEDIUM], c_med);
}

// every segment of the arena, level by level, for parity checks
// (15 floats per segment: t, b1, b2, origin, direction, throughput W and
// an escaped segment's contribution W * E(d), which k_shade added to its
// pixel divided by spp).
constexpr int kSegF = 15;
__global__ void k_dump(WsView W, int32_t* __restrict__ si, float* __restrict__ sf, unsigned long long cap) {
  const WsHeader* H = W.hdr;
  if (H->ring) return;  // hit records of checkpointed renders are not kept
  if (H->mom) return;   // a tape with medium moments has another layout than the one cap was derived for
  const int nl = (int)H->n_levels;
  const unsigned long long total = nl > 0 ? H->level_start[nl] : 0ull;
  const unsigned long long lim = total < cap ? total : cap;
  const int n_scenes = W.th->n;
  for (unsigned long long a = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; a < lim;
       a += (unsigned long long)gridDim.x * blockDim.x) {
    const float4 ro = W.ray_o[a], rd = W.ray_d[a], rw = W.ray_w[a], hh = W.hit[a];
    const uint32_t sample = __float_as_uint(ro.w);
    const int tri = __float_as_int(hh.w);
    si[4 * a + 0] = (int32_t)sample;
    si[4 * a + 1] = __float_as_int(rd.w);
    si[4 * a + 2] = tri;
    si[4 * a + 3] = (int32_t)(W.sflag[a] & SF_FLAG_BITS);
    float3 c = mk(0.f, 0.f, 0.f);
    if (tri < 0) {  // the same lookup as k_shade's, on the segment's own scene
      const SceneEntry& E = W.ent[find_scene(W.th->starts, n_scenes, sample)];
      if (sample >= E.sample_start && (sample - E.sample_start) / (uint32_t)E.spp < E.pix_count) {
        const float3 Ev = env_lookup(E.env, E.env_w, E.env_h, xyz(rd));
        c = mk(rw.x * Ev.x, rw.y * Ev.y, rw.z * Ev.z);
      }
    }
    float* f = sf + kSegF * a;
    f[0] = hh.x; f[1] = hh.y; f[2] = hh.z;
    f[3] = ro.x; f[4] = ro.y; f[5] = ro.z;
    f[6] = rd.x; f[7] = rd.y; f[8] = rd.z;
    f[9] = rw.x; f[10] = rw.y; f[11] = rw.z;
    f[12] = c.x; f[13] = c.y; f[14] = c.z;
  }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
// Launch and scheduling knobs (dt_set_tuning; defined with the C ABI).
extern dt_tuning g_tuning;
// Traversal order of level k from the buckets counted while it was shaded
// into existence, and the clearing of the bucket counters (dt_order.cu).
void launch_order(const WsView& W, int k, int bits, cudaStream_t s);
void launch_order_clear(const WsView& W, int bits, cudaStream_t s);
static int shade_blocks() { return g_tuning.shade_blocks_per_sm * num_sms(); }
static int n_int_of(int32_t nf) { return nf > 1 ? nf - 1 : 1; }

// The traversal is compiled for 2..8 resident CTAs of 256 threads per SM (the
// register budget per thread follows) and for the 2- and 4-wide node
// formats; the tuning picks the variant and the persistent grid is
// trace_blocks_per_sm CTAs per SM.
template <int kWidth, bool kBatch, typename... A>
static void launch_trace_w(int bps, cudaStream_t s, A... a) {
  const int g = bps * num_sms();
  switch (bps) {
    case 1: case 2: case 3: k_trace<3, kWidth, kBatch><<<g, 256, 0, s>>>(a...); break;
    case 4: k_trace<4, kWidth, kBatch><<<g, 256, 0, s>>>(a...); break;
    case 5: k_trace<5, kWidth, kBatch><<<g, 256, 0, s>>>(a...); break;
    default: k_trace<6, kWidth, kBatch><<<g, 256, 0, s>>>(a...); break;
  }
}
static int traversal_limit(int32_t nf) { return 2 * n_int_of(nf) + 8; }

// Writes the scene table (header + entries) into the workspace.
void launch_write_table(const WsView& W, const TableHeader& th, const SceneEntry* entries, int n, cudaStream_t s) {
  ProfScope ps("k_write_table", s);
  for (int first = 0; first < n; first += kEntriesPerChunk) {
    TableChunk c;
    c.first = first;
    c.count = n - first < kEntriesPerChunk ? n - first : kEntriesPerChunk;
    for (int k = 0; k < c.count; ++k) c.e[k] = entries[first + k];
    k_write_table<<<1, 256, 0, s>>>(W.th, th, W.ent, c, first == 0 ? 1 : 0);
  }
}

// Forward of a table of scenes: camera rays of all of them into level 0,
// then per depth one persistent traversal and one shading pass over the
// segments of every scene together.
void launch_forward_table(const TableHeader& th, const SceneEntry* entries, void* ws, unsigned long long cap,
                          unsigned long long ring, bool mom, cudaStream_t s) {
  WsView W = ws_view(ws, cap, ring, mom);
  const int n = th.n;
  cudaMemsetAsync(ws, 0, 1024, s);
  launch_write_table(W, th, entries, n, s);
  uint32_t max_s = 0;
  for (int i = 0; i < n; ++i) {
    const uint32_t ns = entries[i].pix_count * (uint32_t)entries[i].spp;
    if (ns > max_s) max_s = ns;
  }
  int cb = (int)((max_s + 255) / 256);
  if (cb > 4 * num_sms()) cb = 4 * num_sms();
  {
    ProfScope ps("k_camera", s);
    k_camera<<<dim3(cb > 0 ? cb : 1, n), 256, 0, s>>>(W, cap);
  }
  const bool batch = n > 1;
  const SceneEntry& E0 = entries[0];
  const int bps = g_tuning.trace_blocks_per_sm, st = g_tuning.trace_steps, rf = g_tuning.trace_refill;
  // levels after the camera rays are traced bucket by bucket (dt_order.cu);
  // the camera rays keep pixel order, which is coherent
  // (small renders are launch-bound: their levels keep append order)
  const int order_bits = th.n_samples >= (uint32_t)g_tuning.order_min_rays ? g_tuning.trace_order : 0;
  for (int k = 0; k <= th.max_depth; ++k) {
    const int sorted = order_bits && k > 0;
    if (sorted) launch_order(W, k, order_bits, s);
    {
      ProfScope ps("k_trace", s);
      if (g_tuning.bvh_width == 4) {
        if (batch) launch_trace_w<4, true>(bps, s, W, k, st, rf, E0, sorted);
        else launch_trace_w<4, false>(bps, s, W, k, st, rf, E0, sorted);
      } else {
        if (batch) launch_trace_w<2, true>(bps, s, W, k, st, rf, E0, sorted);
        else launch_trace_w<2, false>(bps, s, W, k, st, rf, E0, sorted);
      }
    }
    if (W.mom && th.any_medium) {
      ProfScope ps("k_medium_forward", s);
      const int mb = 8 * num_sms();
      if (th.any_medium == 2) {
        if (batch) k_medium_forward<true, true><<<mb, 256, 0, s>>>(W, k, E0);
        else k_medium_forward<false, true><<<mb, 256, 0, s>>>(W, k, E0);
      } else {
        if (batch) k_medium_forward<true, false><<<mb, 256, 0, s>>>(W, k, E0);
        else k_medium_forward<false, false><<<mb, 256, 0, s>>>(W, k, E0);
      }
    }
    {
      const int bits = k < th.max_depth ? order_bits : 0;
      if (bits) launch_order_clear(W, bits, s);
      ProfScope ps("k_shade", s);
      if (th.any_medium == 2) {
        if (batch) k_shade<true, 2><<<shade_blocks(), kShadeThreads, 0, s>>>(W, k, E0, bits);
        else k_shade<false, 2><<<shade_blocks(), kShadeThreads, 0, s>>>(W, k, E0, bits);
      } else if (th.any_medium) {
        if (batch) k_shade<true, 1><<<shade_blocks(), kShadeThreads, 0, s>>>(W, k, E0, bits);
        else k_shade<false, 1><<<shade_blocks(), kShadeThreads, 0, s>>>(W, k, E0, bits);
      } else {
        if (batch) k_shade<true, 0><<<shade_blocks(), kShadeThreads, 0, s>>>(W, k, E0, bits);
        else k_shade<false, 0><<<shade_blocks(), kShadeThreads, 0, s>>>(W, k, E0, bits);
      }
    }
  }
}

// One table entry for a scene as given at the C ABI.
SceneEntry make_entry(const dt_scene& sc, const dt_views& vw, const dt_params& p, float* out) {
  SceneEntry e;
  memset(&e, 0, sizeof(e));
  BvhView B = bvh_view(sc.d_bvh, sc.nf);
  e.V = sc.d_V; e.F = sc.d_F; e.N = sc.d_N; e.ior = sc.d_ior; e.sigma = sc.d_sigma; e.env = sc.d_env;
  e.node2 = B.node2; e.node4 = B.node4; e.tris = B.tris; e.bh = B.hdr;
  e.cams = vw.d_cams; e.out = out;
  e.seed = p.seed;
  e.nv = sc.nv; e.nf = sc.nf; e.env_w = sc.env_w; e.env_h = sc.env_h;
  e.n_views = vw.n_views; e.width = vw.width; e.height = vw.height; e.spp = p.spp;
  e.max_depth = p.max_depth; e.jitter = p.jitter; e.max_iter = traversal_limit(sc.nf);
  e.t_min = p.t_min;
  e.pix_count = (uint32_t)vw.n_views * (uint32_t)vw.width * (uint32_t)vw.height;
  e.denv = sc.d_grad_env;
  if (sc.medium && sc.medium->d_mu) {
    const dt_medium& M = *sc.medium;
    e.mu = reinterpret_cast<const float4*>(M.d_mu);
    e.dmu = reinterpret_cast<float4*>(M.d_grad_mu);
    e.gnx = M.nx; e.gny = M.ny; e.gnz = M.nz;
    e.glo_x = M.lo[0]; e.glo_y = M.lo[1]; e.glo_z = M.lo[2];
    e.gscale_x = (float)(M.nx - 1) / (M.hi[0] - M.lo[0]);
    e.gscale_y = (float)(M.ny - 1) / (M.hi[1] - M.lo[1]);
    e.gscale_z = (float)(M.nz - 1) / (M.hi[2] - M.lo[2]);
    e.gstep = M.step;
    if (M.levels > 0) {  // hash texture: the dense fields stay unused
      const uint32_t T = 1u << M.log2_table;
      e.glevels = M.levels;
      e.gentries = (uint32_t)M.levels * T;
      for (int l = 0; l < M.levels; ++l) {
        const int r = M.res[l];
        GridLevel& L = e.glev[l];
        L.n = r;
        L.mask = (double)r * r * r > (double)T ? T - 1u : 0u;
        L.off = (uint32_t)l * T;
        L.sx = (float)(r - 1) / (M.hi[0] - M.lo[0]);
        L.sy = (float)(r - 1) / (M.hi[1] - M.lo[1]);
        L.sz = (float)(r - 1) / (M.hi[2] - M.lo[2]);
      }
    } else {
      e.gentries = (uint32_t)((size_t)M.nx * M.ny * M.nz);
    }
  }
  return e;
}

// Fills sample/face offsets of the entries and the table header.
void finish_table(SceneEntry* entries, int n, TableHeader& th) {
  memset(&th, 0, sizeof(th));
  th.n = n;
  uint32_t s = 0, f = 0;
  int md = 0;
  for (int i = 0; i < n; ++i) {
    entries[i].sample_start = s;
    entries[i].face_start = f;
    th.starts[i] = s;
    th.face_starts[i] = f;
    s += entries[i].pix_count * (uint32_t)entries[i].spp;
    f += (uint32_t)entries[i].nf;
    if (entries[i].max_depth > md) md = entries[i].max_depth;
    if (entries[i].mu && th.any_medium < 2) th.any_medium = entries[i].glevels > 0 ? 2 : 1;
    if (entries[i].denv) th.any_env_grad = 1;
  }
  th.starts[n] = s;
  th.face_starts[n] = f;
  th.n_samples = s;
  th.n_faces = f;
  th.max_depth = md;
}

void launch_dump(const void* ws, unsigned long long cap, int32_t* si, float* sf, unsigned long long n,
                 cudaStream_t s) {
  WsView W = ws_view(ws, cap, 0);  // a checkpointed render's dump returns at once (k_dump)
  k_dump<<<4 * num_sms(), 256, 0, s>>>(W, si, sf, n);
}

void launch_closest_hit(const void* bvh, int32_t nf, const float* o, const float* d, const int32_t* src, int32_t n,
                        float tmin, int32_t* tri, float* tbb, cudaStream_t s) {
  BvhView B = bvh_view(bvh, nf);
  int b = (n + 127) / 128;
  if (b > 8 * num_sms()) b = 8 * num_sms();
  k_closest_hit_rays<<<b > 0 ? b : 1, 128, 0, s>>>(B.node2, B.tris, o, d, src, n, B.hdr, tmin,
                                                    traversal_limit(nf), tri, tbb);
}

}  // namespace dt

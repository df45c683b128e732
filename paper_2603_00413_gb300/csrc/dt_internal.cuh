// Internal definitions shared by the CUDA translation units of libdifftrans:
// float3 arithmetic, the device layouts of the BVH buffer and of the render
// workspace (the segment "tape"), segment and status flag bits, and the
// launch helpers.  FP32 throughout; no fast-math approximations (divisions
// and square roots are IEEE round-to-nearest).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/difftrans.h"

namespace dt {

// ---------------------------------------------------------------------------
// float3 arithmetic
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ float3 mk(float x, float y, float z) { return make_float3(x, y, z); }
__host__ __device__ __forceinline__ float3 operator+(float3 a, float3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
__host__ __device__ __forceinline__ float3 operator-(float3 a, float3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
__host__ __device__ __forceinline__ float3 operator-(float3 a) { return mk(-a.x, -a.y, -a.z); }
__host__ __device__ __forceinline__ float3 operator*(float3 a, float s) { return mk(a.x * s, a.y * s, a.z * s); }
__host__ __device__ __forceinline__ float3 operator*(float s, float3 a) { return mk(a.x * s, a.y * s, a.z * s); }
__host__ __device__ __forceinline__ float3 mul(float3 a, float3 b) { return mk(a.x * b.x, a.y * b.y, a.z * b.z); }
__host__ __device__ __forceinline__ float dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__host__ __device__ __forceinline__ float3 cross(float3 a, float3 b) {
  return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__host__ __device__ __forceinline__ float len(float3 a) { return sqrtf(dot(a, a)); }
// cross product with every product rounded before the subtraction (no fused
// multiply-add): exactly zero for parallel inputs such as a x a, which a
// contracted form is not (it keeps one product's rounding error)
__device__ __forceinline__ float3 cross_rn(float3 a, float3 b) {
  return mk(__fsub_rn(__fmul_rn(a.y, b.z), __fmul_rn(a.z, b.y)), __fsub_rn(__fmul_rn(a.z, b.x), __fmul_rn(a.x, b.z)),
            __fsub_rn(__fmul_rn(a.x, b.y), __fmul_rn(a.y, b.x)));
}
__host__ __device__ __forceinline__ float3 normalize(float3 a) {
  float n = len(a);
  return mk(a.x / n, a.y / n, a.z / n);
}
__device__ __forceinline__ float3 xyz(float4 v) { return mk(v.x, v.y, v.z); }
__device__ __forceinline__ float3 load3(const float* p) { return mk(p[0], p[1], p[2]); }

// ---------------------------------------------------------------------------
// segment flags (same bit meaning as the parity dump in difftrans.h)
// ---------------------------------------------------------------------------
enum : uint32_t {
  SF_INSIDE = 4u,
  SF_TIR = 8u,
  SF_BACKFACING = 16u,
  SF_DISCARDED = 128u,
  SF_MISS = 512u,
  SF_FLAG_BITS = 0xffffu,  // the event bits; above them the refracted child's offset
};
constexpr int kRefractShift = 16;  // sflag >> 16 = refracted child index - reflected child index

// device status bits (render workspace header)
enum : uint32_t {
  ST_QUEUE_OVERFLOW = 1u,
  ST_STACK_OVERFLOW = 2u,
};

constexpr int kMaxLevels = 32;
constexpr int kMaxDepth = 30;
constexpr int kTraceStack = 64;

// ---------------------------------------------------------------------------
// BVH buffer.  A binary LBVH (Karras) is built and refitted; the traversal
// reads a 4-wide BVH derived from it: every binary node at even depth is a
// 4-wide node whose children are its grandchildren (a leaf child stays one
// child, so a node has 2 to 4 children).
//  - bin_child[j] = (left, right) of binary internal node j; a child >= 0 is
//    internal, < 0 is leaf ~child (a one-triangle mesh has one node whose two
//    children are both leaf 0).  parent[] holds the parent of internal
//    node j at j and of leaf i at n_int + i.
//  - box_int[2j], box_int[2j+1] = (lo, hi) of binary node j;
//    box_leaf[2i], box_leaf[2i+1] = (lo, hi) of leaf i.
//  - node4[8m .. 8m+7]: 4-wide node m as float4 rows (one component per
//    child): lo.x, hi.x, lo.y, hi.y, lo.z, hi.z, child refs (int bits: >= 0
//    node4 index, < 0 leaf ~i, kNoChild empty with an empty box), and the
//    binary sources of the four boxes (same encoding, for the refit).
//  - bin_to4[j] = node4 index of binary node j (even depth) or -1.
//  - node2[4j .. 4j+3]: binary node j for the 2-wide traversal: child-0 box
//    (lo.x, hi.x, lo.y, hi.y), child-1 box (same), (c0 lo.z, hi.z, c1 lo.z,
//    hi.z), (child0, child1) as int bits (leaf ~i, kNoChild empty).
//  - tris[3i..3i+2] = leaf i's triangle: (v0, id), (e1, 0), (e2, 0).
//  - leaf_tri[i] = triangle of leaf i.
// ---------------------------------------------------------------------------
constexpr int kNoChild = (int)0x80000000;

struct BvhHeader {
  int32_t nf;
  int32_t n_int;    // binary internal nodes = max(nf - 1, 1)
  int32_t n4;       // 4-wide nodes (written on the device)
  int32_t corrupt;  // set by the build's validation pass when a reference is out of range
};

struct BvhView {
  BvhHeader* hdr;
  int2* bin_child;   // [n_int]
  int32_t* parent;   // [n_int + nf]
  float4* box_int;   // [2 n_int]
  float4* box_leaf;  // [2 nf]
  float4* node4;     // [8 n_int] (at most n_int 4-wide nodes)
  float4* node2;     // [4 n_int]
  int32_t* bin_to4;  // [n_int]
  float4* tris;      // [3 nf]
  int32_t* leaf_tri; // [nf]
};

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct BvhLayout {
  size_t off_child, off_parent, off_box_int, off_box_leaf, off_node4, off_node2, off_bin_to4, off_tris, off_leaf,
      total;
  __host__ __device__ explicit BvhLayout(int32_t nf) {
    const size_t n_int = nf > 1 ? (size_t)nf - 1 : 1;
    size_t o = 256;
    auto take = [&](size_t bytes) { size_t r = o; o = align_up(o + bytes, 256); return r; };
    off_node4 = take(n_int * 8 * sizeof(float4));
    off_node2 = take(n_int * 4 * sizeof(float4));
    off_tris = take((size_t)nf * 3 * sizeof(float4));
    off_child = take(n_int * sizeof(int2));
    off_parent = take((n_int + (size_t)nf) * sizeof(int32_t));
    off_box_int = take(n_int * 2 * sizeof(float4));
    off_box_leaf = take((size_t)nf * 2 * sizeof(float4));
    off_bin_to4 = take(n_int * sizeof(int32_t));
    off_leaf = take((size_t)nf * sizeof(int32_t));
    total = o;
  }
};

__host__ __device__ inline BvhView bvh_view(const void* base, int32_t nf) {
  BvhLayout L(nf);
  char* b = (char*)base;
  return BvhView{(BvhHeader*)b, (int2*)(b + L.off_child), (int32_t*)(b + L.off_parent),
                 (float4*)(b + L.off_box_int), (float4*)(b + L.off_box_leaf), (float4*)(b + L.off_node4),
                 (float4*)(b + L.off_node2), (int32_t*)(b + L.off_bin_to4), (float4*)(b + L.off_tris),
                 (int32_t*)(b + L.off_leaf)};
}

// ---------------------------------------------------------------------------
// Render workspace: a header, then the segment arena.  Level k occupies
// [level_start[k], level_start[k] + count(k)).  Per segment i:
//   ray_o[i] = (origin xyz, sample index as int bits)
//   ray_d[i] = (direction xyz, heap node id as int bits)
//   ray_w[i] = (throughput rgb, triangle the ray leaves from, or -1)
//   hit[i]   = (t, b1, b2, hit triangle or -1)
//   child[i] = arena index of the reflected child, -1 when it has none
//   sflag[i] = SF_* bits; bits 16-31: the refracted child's index minus
//              child[i] (0 when there is none: total internal reflection)
// ---------------------------------------------------------------------------
struct WsHeader {
  uint32_t status;
  uint32_t n_levels;
  unsigned long long capacity;
  unsigned long long seg_needed;
  uint32_t level_count[kMaxLevels];  // appended (may exceed what fits)
  uint32_t level_start[kMaxLevels];
  uint32_t fetch[kMaxLevels];        // work-fetch cursors of the trace kernels
  unsigned long long counters[16];   // see CNT_*
  uint32_t ring;                     // level capacity of the hit ring (tape_mode 1), 0 = every hit kept
  uint32_t mom;                      // 1: the medium moments of tape_mode 2 follow the hit records
};

enum { CNT_HITS = 0, CNT_MISSES, CNT_DISCARDED, CNT_BACKFACING, CNT_TIR, CNT_NODES, CNT_TRIS, CNT_MEDIUM };

// ---------------------------------------------------------------------------
// Scene table: every render (one scene or a batch) reads its scenes from a
// table in the workspace, written by a kernel whose parameters carry the
// entries.  Segments find their scene by binary search of their sample index
// in starts[] (faces by face_starts[] for the per-face kernels).
// ---------------------------------------------------------------------------
constexpr int kMaxBatch = 256;
constexpr int kEntriesPerChunk = 24;  // table entries per writing launch (kernel-parameter space)

// One level of a hash texture (dt_medium levels > 0).
constexpr int kMaxGridLevels = 16;
struct alignas(16) GridLevel {
  int32_t n;         // nodes per axis
  uint32_t mask;     // hashed level: entries per level - 1; 0: dense indexing (k n + j) n + i
  uint32_t off;      // first table entry of the level
  float sx, sy, sz;  // nodes per unit length minus the fencepost ((n - 1) / (hi - lo))
  int32_t pad[2];
};
static_assert(sizeof(GridLevel) == 32, "levels are read as two 16-byte vectors");

struct SceneEntry {
  const float* V;
  const int32_t* F;
  const float* N;
  const float* ior;
  const float* sigma;
  const float* env;
  const float4* node2;
  const float4* node4;
  const float4* tris;
  const BvhHeader* bh;
  const float* cams;
  float* out;
  const float* grad_out;  // backward only
  float* dV;
  float* dior;
  float* dsigma;
  float* dN;
  unsigned long long seed;
  int32_t nv, nf, env_w, env_h;
  int32_t n_views, width, height, spp;
  int32_t max_depth, jitter, max_iter, pad0;
  float t_min;
  uint32_t sample_start, face_start, pix_count;
  // absorption grid (dt_medium; mu == nullptr: none): node values, their
  // gradient (backward, may be nullptr), node counts, box origin, nodes per
  // unit length minus the fencepost ((n - 1) / (hi - lo)), step length
  const float4* mu;
  float4* dmu;
  int32_t gnx, gny, gnz;
  float glo_x, glo_y, glo_z;
  float gscale_x, gscale_y, gscale_z;
  float gstep;
  float* denv;  // backward: gradient of the environment texels (nullptr: not computed)
  // hash texture (glevels > 0; mu then holds the levels' tables and the
  // dense fields above are unused); gentries = float4 entries of mu
  int32_t glevels;
  uint32_t gentries;
  GridLevel glev[kMaxGridLevels];
};

struct TableHeader {
  int32_t n;
  int32_t max_depth;
  int32_t any_medium;  // some scene of the table has an absorption grid (2: a hash texture)
  int32_t any_env_grad;  // some scene of the table wants its environment gradient
  uint32_t n_samples;
  uint32_t n_faces;
  uint32_t starts[kMaxBatch + 1];
  uint32_t face_starts[kMaxBatch + 1];
};

struct TableView {
  const TableHeader* th;
  const SceneEntry* e;
};

constexpr size_t kTableBytes =
    ((sizeof(TableHeader) + 255) / 256) * 256 + ((kMaxBatch * sizeof(SceneEntry) + 255) / 256) * 256;

// Traversal order of a level (dt_order.cu): a counting sort over at most
// 2^kOrderBits buckets, whose counters (and at most 1024 span totals of
// their scan) take a fixed region of the workspace.
constexpr int kOrderBits = 22;
constexpr uint32_t kOrderCounters = 1u << kOrderBits;
constexpr size_t kOrderBytes = (((size_t)kOrderCounters + 1024) * sizeof(uint32_t) + 255) / 256 * 256;

// index i with starts[i] <= x < starts[i+1] (n >= 1)
__device__ __forceinline__ int find_scene(const uint32_t* starts, int n, uint32_t x) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(starts + mid) <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

struct WsView {
  WsHeader* hdr;
  TableHeader* th;
  SceneEntry* ent;
  float4* ray_o;
  float4* ray_d;
  float4* ray_w;
  float4* hit;
  int32_t* child;
  uint32_t* sflag;
  unsigned long long cap;
  uint32_t ring;  // 0: hit[a] for arena index a; else hit[(k & 1) ring + i] for position i in level k
  uint32_t* order_count;  // traversal order: kOrderCounters bucket counters, then the scan's span totals
  float* mom;     // tape_mode 2: kMomFloats arrays of cap floats (medium moments, see below); else null
};

// tape_mode 2 keeps, for every interior segment of a scene with an absorption
// grid or hash texture, the optical depth of the medium over the segment and
// its derivatives, written by the forward's medium pass, so that neither the
// shading pass nor the backward marches the medium again.  Array j of the
// kMomFloats (mom[j cap + a] for arena index a): 0-2 S (per channel), 3-5
// dS/dt, 6-14 dS_c/do_x..z (c = 0..2, row-major), 15-23 dS_c/dd_x..z.
// S_0 = NaN marks a segment the pass did not march (it found it entering).
constexpr int kMomFloats = 24;
constexpr int kMomS = 0, kMomDt = 3, kMomDo = 6, kMomDd = 15;

// Where the hit record of position i of level k (arena index a) lives.
__device__ __forceinline__ size_t hit_slot(const WsView& W, int k, uint32_t a, uint32_t i) {
  return W.ring ? (size_t)(k & 1) * W.ring + i : (size_t)a;
}

// The hit records of level k (arena start `start`) seen as 32-bit words.
// Until level k is traced the first n words hold each segment's
// traversal-order bucket (written with the segment by the shading pass of
// level k-1).
__device__ __forceinline__ uint32_t* level_buckets(const WsView& W, int k, uint32_t start) {
  return reinterpret_cast<uint32_t*>(W.hit + (W.ring ? (size_t)(k & 1) * W.ring : (size_t)start));
}

// Traversal-order key of a ray: the direction octant in bits 21-23 above the
// 21-bit Morton code of its origin on a 128^3 grid over the scene's bounding
// box (lo, and 128 / extent per axis).  Rays that share the octant and leave
// nearby points take similar paths through the BVH.
__device__ __forceinline__ uint32_t spread7(uint32_t v) {
  v = (v | (v << 8)) & 0x0000F00Fu;
  v = (v | (v << 4)) & 0x000C30C3u;
  v = (v | (v << 2)) & 0x00249249u;
  return v;
}
__device__ __forceinline__ uint32_t cell7(float x, float lo, float scale) {
  return (uint32_t)fminf(fmaxf((x - lo) * scale, 0.0f), 127.0f);
}
__device__ __forceinline__ uint32_t ray_order_key(float3 o, float3 d, float3 lo, float3 scale) {
  const uint32_t oct = ((d.x < 0.0f) ? 4u : 0u) | ((d.y < 0.0f) ? 2u : 0u) | ((d.z < 0.0f) ? 1u : 0u);
  return (oct << 21) | (spread7(cell7(o.x, lo.x, scale.x)) << 2) | (spread7(cell7(o.y, lo.y, scale.y)) << 1) |
         spread7(cell7(o.z, lo.z, scale.z));
}
// Bucket of a key with `bits` bits (12..kOrderBits): its top bits, below the
// scene index (8 bits) in a batch.
__device__ __forceinline__ uint32_t order_bucket(uint32_t key24, int bits, bool batch, uint32_t scene) {
  return batch ? (scene << (bits - 8)) | (key24 >> (32 - bits)) : key24 >> (24 - bits);
}
// Counts a child in its bucket and stores the bucket at its position p of
// the next level; b == ~0u: no child.
__device__ __forceinline__ void order_count_child(uint32_t* count, uint32_t* kb, uint32_t b, uint32_t p) {
  if (b != ~0u) {
    kb[p] = b;
    atomicAdd(count + b, 1u);
  }
}

// Bounding box of a scene from its binary BVH root (node 0): lo and the
// 128-cells-per-axis scale of ray_order_key.
__device__ __forceinline__ void scene_order_box(const float4* __restrict__ node2, float3& lo, float3& scale) {
  const float4 a = __ldg(node2), b = __ldg(node2 + 1), c = __ldg(node2 + 2);
  lo = mk(fminf(a.x, b.x), fminf(a.z, b.z), fminf(c.x, c.z));
  const float3 hi = mk(fmaxf(a.y, b.y), fmaxf(a.w, b.w), fmaxf(c.y, c.w));
  scale = mk(128.0f / fmaxf(hi.x - lo.x, 1e-30f), 128.0f / fmaxf(hi.y - lo.y, 1e-30f),
             128.0f / fmaxf(hi.z - lo.z, 1e-30f));
}

// Arena layout; the hit records come last, so every other offset depends on
// the segment capacity only.  ring = 0: one hit per segment; else a ring of
// two levels of `ring` hits.
struct WsLayout {
  size_t off_table, off_order, off_o, off_d, off_w, off_child, off_flag, off_hit, off_mom, total;
  __host__ __device__ explicit WsLayout(unsigned long long cap, unsigned long long ring = 0, bool mom = false) {
    off_table = 1024;
    off_order = off_table + kTableBytes;
    off_o = off_order + kOrderBytes;
    off_d = align_up(off_o + cap * sizeof(float4), 256);
    off_w = align_up(off_d + cap * sizeof(float4), 256);
    off_child = align_up(off_w + cap * sizeof(float4), 256);
    off_flag = align_up(off_child + cap * sizeof(int32_t), 256);
    off_hit = align_up(off_flag + cap * sizeof(uint32_t), 256);
    off_mom = align_up(off_hit + (ring ? 2 * ring : cap) * sizeof(float4), 256);
    total = align_up(off_mom + (mom ? cap * kMomFloats * sizeof(float) : 0), 256);
  }
};
static_assert(sizeof(WsHeader) <= 1024, "header must fit its slot");

__host__ __device__ inline WsView ws_view(const void* base, unsigned long long cap, unsigned long long ring = 0,
                                          bool mom = false) {
  WsLayout L(cap, ring, mom);
  char* b = (char*)base;
  TableHeader* th = (TableHeader*)(b + L.off_table);
  SceneEntry* ent = (SceneEntry*)(b + L.off_table + ((sizeof(TableHeader) + 255) / 256) * 256);
  return WsView{(WsHeader*)b, th, ent, (float4*)(b + L.off_o), (float4*)(b + L.off_d), (float4*)(b + L.off_w),
                (float4*)(b + L.off_hit), (int32_t*)(b + L.off_child), (uint32_t*)(b + L.off_flag), cap,
                (uint32_t)ring, (uint32_t*)(b + L.off_order), mom ? (float*)(b + L.off_mom) : nullptr};
}

// Segments of level k that fit in the arena (and in the hit ring, if any).
__device__ __forceinline__ uint32_t level_size(const WsHeader* h, int k) {
  const unsigned long long start = h->level_start[k];
  if (start >= h->capacity) return 0;
  const unsigned long long room = h->capacity - start;
  unsigned long long n = h->level_count[k];
  if (n > room) n = room;
  if (h->ring && n > h->ring) n = h->ring;
  return (uint32_t)n;
}

// ---------------------------------------------------------------------------
// warp helpers
// ---------------------------------------------------------------------------
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ void warp_add_u64(unsigned long long* dst, unsigned v) {
  unsigned s = __reduce_add_sync(kFull, v);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(dst, (unsigned long long)s);
}

__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// PCG hash (Jarzynski & Olano, "Hash Functions for GPU Rendering", JCGT 2020)
__host__ __device__ __forceinline__ uint32_t pcg_hash(uint32_t v) {
  uint32_t state = v * 747796405u + 2891336453u;
  uint32_t word = ((state >> ((state >> 28u) + 4u)) ^ state) * 277803737u;
  return (word >> 22u) ^ word;
}

// ---------------------------------------------------------------------------
// host-side helpers (defined in dt_api.cu)
// ---------------------------------------------------------------------------
dt_status set_error(dt_status code, const char* fmt, ...);
dt_status check_launch(const char* what);
int num_sms();
void launch_scan_exclusive(uint32_t* a, int32_t m, cudaStream_t s);  // dt_bvh.cu

// Per-kernel event timing (dt_profile_enable).  Scoped: records a start event
// on construction and a stop event on destruction when profiling is on.
struct ProfScope {
  int slot;
  cudaStream_t stream;
  ProfScope(const char* name, cudaStream_t s);
  ~ProfScope();
};

}  // namespace dt

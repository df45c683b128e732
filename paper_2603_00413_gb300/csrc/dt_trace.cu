// Forward wavefront of the recursive tracer (DiffTrans Sec. 3.4 "Recursive
// Ray Tracing", steps 1-5): camera rays into level 0, then per depth k a
// persistent closest-hit traversal of the LBVH and a shading pass that
// accumulates escaped rays into the image and appends the Fresnel-weighted
// reflected and refracted children to level k+1.
#include <cuda_runtime.h>
#include <stdint.h>

#include "dt_internal.cuh"
#include "dt_shade.cuh"

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

__global__ void k_camera(WsView W, const float* __restrict__ cams, int n_views, int width, int height, int spp,
                         int jitter, uint64_t seed, unsigned long long capacity, int max_depth) {
  const uint32_t npix = (uint32_t)width * (uint32_t)height;
  const uint32_t n0 = (uint32_t)n_views * npix * (uint32_t)spp;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    W.hdr->capacity = capacity;
    W.hdr->level_count[0] = n0;
    W.hdr->level_start[0] = 0;
    W.hdr->n_views = n_views; W.hdr->width = width; W.hdr->height = height;
    W.hdr->spp = spp; W.hdr->max_depth = max_depth;
  }
  for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < n0; g += gridDim.x * blockDim.x) {
    const uint32_t s = g % (uint32_t)spp;
    const uint32_t gp = g / (uint32_t)spp;
    const uint32_t view = gp / npix, p = gp % npix;
    float jx = 0.5f, jy = 0.5f;
    if (jitter) jitter_offset(seed, view, p, s, jx, jy);
    float3 o, d;
    camera_ray(cams + 10 * view, width, height, (float)(p % width) + jx, (float)(p / width) + jy, o, d);
    W.ray_o[g] = make_float4(o.x, o.y, o.z, __uint_as_float(g));
    W.ray_d[g] = make_float4(d.x, d.y, d.z, __uint_as_float(1u));
    W.ray_w[g] = make_float4(1.f, 1.f, 1.f, __int_as_float(-1));
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

// A tree traversal visits every internal node at most once, so more than
// max_iter = 2 n_int + 8 steps means a corrupt hierarchy: give up and flag it.
__device__ __forceinline__ ClosestHit closest_hit(const float4* __restrict__ nodes, const float4* __restrict__ tris,
                                                  float3 o, float3 d, int src, float tmin, int max_iter,
                                                  uint32_t& nvis, uint32_t& ntest, bool& overflow) {
  ClosestHit h{INFINITY, 0.f, 0.f, -1};
  const float3 idir = mk(safe_inv(d.x), safe_inv(d.y), safe_inv(d.z));
  int stack[kTraceStack];
  int sp = 0;
  int node = 0;
  for (int it = 0;; ++it) {
    if (it >= max_iter) {
      overflow = true;
      break;
    }
    const float4* N = nodes + 4 * node;
    const float4 n0 = __ldg(N), n1 = __ldg(N + 1), n2 = __ldg(N + 2);
    const int4 n3 = __ldg(reinterpret_cast<const int4*>(N) + 3);
    ++nvis;
    float tn0, tn1;
    bool h0 = slab(o, idir, n0.x, n0.y, n0.z, n0.w, n2.x, n2.y, tmin, h.t, tn0);
    bool h1 = slab(o, idir, n1.x, n1.y, n1.z, n1.w, n2.z, n2.w, tmin, h.t, tn1);
    if (h0 && n3.x < 0) { test_leaf(tris, ~n3.x, o, d, src, tmin, h, ntest); h0 = false; }
    if (h1 && n3.y < 0) { test_leaf(tris, ~n3.y, o, d, src, tmin, h, ntest); h1 = false; }
    if (h0 && h1) {
      int nearc = n3.x, farc = n3.y;
      if (tn1 < tn0) { nearc = n3.y; farc = n3.x; }
      if (sp < kTraceStack) stack[sp++] = farc; else overflow = true;
      node = nearc;
    } else if (h0) {
      node = n3.x;
    } else if (h1) {
      node = n3.y;
    } else {
      if (sp == 0) break;
      node = stack[--sp];
    }
  }
  return h;
}

// Persistent traversal of level k: warps take 32 segments at a time from a
// shared cursor until the level is exhausted.
__global__ void __launch_bounds__(256) k_trace(WsView W, const float4* __restrict__ nodes,
                                               const float4* __restrict__ tris, int k, float tmin, int max_iter) {
  WsHeader* H = W.hdr;
  const uint32_t n = level_size(H, k);
  const uint32_t start = H->level_start[k];
  const uint32_t lane = threadIdx.x & 31;
  uint32_t nvis = 0, ntest = 0;
  bool overflow = false;
  while (true) {
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(&H->fetch[k], 32u);
    base = __shfl_sync(kFull, base, 0);
    if (base >= n) break;
    const uint32_t i = base + lane;
    if (i < n) {
      const uint32_t a = start + i;
      const float4 ro = W.ray_o[a], rd = W.ray_d[a], rw = W.ray_w[a];
      const ClosestHit h = closest_hit(nodes, tris, xyz(ro), xyz(rd), __float_as_int(rw.w), tmin, max_iter, nvis,
                                       ntest, overflow);
      W.hit[a] = h.tri >= 0 ? make_float4(h.t, h.b1, h.b2, __int_as_float(h.tri))
                            : make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
    }
  }
  warp_add_u64(&H->counters[CNT_NODES], nvis);
  warp_add_u64(&H->counters[CNT_TRIS], ntest);
  if (__any_sync(kFull, overflow) && lane == 0) atomicOr(&H->status, ST_STACK_OVERFLOW);
}

// Closest hit of arbitrary rays (tooling and tests).
__global__ void k_closest_hit_rays(const float4* __restrict__ nodes, const float4* __restrict__ tris,
                                   const float* __restrict__ o, const float* __restrict__ d,
                                   const int32_t* __restrict__ src, int32_t n, float tmin, int max_iter,
                                   int32_t* __restrict__ tri, float* __restrict__ tbb) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    uint32_t nv = 0, nt = 0;
    bool ovf = false;
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
struct SceneDev {
  const float* V;
  const int32_t* F;
  const float* N;
  const float* ior;
  const float* sigma;
  const float* env;
  int env_w, env_h;
};

__global__ void __launch_bounds__(256) k_shade(WsView W, SceneDev S, int k, int max_depth, int spp,
                                               uint32_t n_pix, float* __restrict__ img) {
  const float inv_spp = 1.0f / (float)spp;
  WsHeader* H = W.hdr;
  const uint32_t n = level_size(H, k);
  const uint32_t start = H->level_start[k];
  const uint32_t next_start = start + n;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    H->level_start[k + 1] = next_start;
    if (n) H->n_levels = (uint32_t)(k + 1);
  }
  const float ior = __ldg(S.ior);
  const float3 sigma = mk(__ldg(S.sigma), __ldg(S.sigma + 1), __ldg(S.sigma + 2));
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t warps = gridDim.x * blockDim.x / 32;
  uint32_t c_hit = 0, c_miss = 0, c_disc = 0, c_back = 0, c_tir = 0;
  bool overflow = false;
  for (uint32_t wb = (blockIdx.x * blockDim.x + threadIdx.x) / 32 * 32; wb < n; wb += warps * 32) {
    const uint32_t i = wb + lane;
    const uint32_t a = start + i;
    int nchild = 0;
    float4 co = make_float4(0.f, 0.f, 0.f, 0.f), cdr = co, cwr = co, cdt = co, cwt = co;
    if (i < n) {
      const float4 ro = W.ray_o[a], rd = W.ray_d[a], rw = W.ray_w[a], hh = W.hit[a];
      const int tri = __float_as_int(hh.w);
      const float3 d = xyz(rd);
      uint32_t fl = 0;
      if (tri < 0) {  // step 3: no intersection -> environment
        fl = SF_MISS;
        ++c_miss;
        const uint32_t pix = __float_as_uint(ro.w) / (uint32_t)spp;
        if (pix < n_pix) {  // dead records (see below) carry an out-of-range sample index
          const float3 E = env_lookup(S.env, S.env_w, S.env_h, d);
          float* dst = img + 3 * (size_t)pix;
          atomicAdd(dst + 0, rw.x * E.x * inv_spp);
          atomicAdd(dst + 1, rw.y * E.y * inv_spp);
          atomicAdd(dst + 2, rw.z * E.z * inv_spp);
        }
      } else {
        ++c_hit;
        const int i0 = __ldg(S.F + 3 * tri), i1 = __ldg(S.F + 3 * tri + 1), i2 = __ldg(S.F + 3 * tri + 2);
        const float3 v0 = load3(S.V + 3 * i0), v1 = load3(S.V + 3 * i1), v2 = load3(S.V + 3 * i2);
        if (k >= max_depth) {  // step 1: the depth limit: contributes nothing
          const float3 ng = cross(v1 - v0, v2 - v0);
          fl = SF_DISCARDED | (dot(d, ng) < 0.0f ? 0u : SF_INSIDE);
          ++c_disc;
        } else {
          HitShade h;
          shade_hit(xyz(ro), d, hh.x, hh.y, hh.z, v0, v1, v2, load3(S.N + 3 * i0), load3(S.N + 3 * i1),
                    load3(S.N + 3 * i2), ior, sigma, h);
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
            if (!h.tir) {
              cdt = make_float4(h.wt.x, h.wt.y, h.wt.z, __uint_as_float(2u * node + 1u));
              cwt = make_float4(Wt.x * h.T, Wt.y * h.T, Wt.z * h.T, __int_as_float(tri));
              nchild = 2;
            }
          }
        }
      }
      W.sflag[a] = fl;
    }
    // warp-aggregated append of the children to level k+1
    int incl = nchild;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(kFull, incl, o);
      if ((int)lane >= o) incl += v;
    }
    const int total = __shfl_sync(kFull, incl, 31);
    uint32_t base = 0;
    if (lane == 0 && total > 0) base = atomicAdd(&H->level_count[k + 1], (uint32_t)total);
    base = __shfl_sync(kFull, base, 0);
    if (i < n) {
      int32_t ch = -1;
      if (nchild > 0) {
        const unsigned long long j = (unsigned long long)next_start + base + (uint32_t)(incl - nchild);
        if (j + (unsigned long long)nchild <= H->capacity) {
          ch = (int32_t)j;
          W.ray_o[j] = co; W.ray_d[j] = cdr; W.ray_w[j] = cwr;
          if (nchild == 2) { W.ray_o[j + 1] = co; W.ray_d[j + 1] = cdt; W.ray_w[j + 1] = cwt; }
        } else {
          overflow = true;
          // a pair that straddles the end of the arena: the slot that still
          // fits gets an inert record (zero direction, no pixel) so nothing
          // below the capacity is ever left unwritten
          if (j < H->capacity) {
            W.ray_o[j] = make_float4(0.f, 0.f, 0.f, __uint_as_float(0xffffffffu));
            W.ray_d[j] = make_float4(0.f, 0.f, 0.f, __uint_as_float(0u));
            W.ray_w[j] = make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
          }
        }
      }
      W.child[a] = ch;
    }
  }
  warp_add_u64(&H->counters[CNT_HITS], c_hit);
  warp_add_u64(&H->counters[CNT_MISSES], c_miss);
  warp_add_u64(&H->counters[CNT_DISCARDED], c_disc);
  warp_add_u64(&H->counters[CNT_BACKFACING], c_back);
  warp_add_u64(&H->counters[CNT_TIR], c_tir);
  if (__any_sync(kFull, overflow) && lane == 0) atomicOr(&H->status, ST_QUEUE_OVERFLOW);
}

// every segment of the arena, level by level, for parity checks
__global__ void k_dump(WsView W, int32_t* __restrict__ si, float* __restrict__ sf, unsigned long long cap) {
  const WsHeader* H = W.hdr;
  const int nl = (int)H->n_levels;
  const unsigned long long total = nl > 0 ? H->level_start[nl] : 0ull;
  const unsigned long long lim = total < cap ? total : cap;
  for (unsigned long long a = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; a < lim;
       a += (unsigned long long)gridDim.x * blockDim.x) {
    const float4 ro = W.ray_o[a], rd = W.ray_d[a], hh = W.hit[a];
    si[4 * a + 0] = __float_as_int(ro.w);
    si[4 * a + 1] = __float_as_int(rd.w);
    si[4 * a + 2] = __float_as_int(hh.w);
    si[4 * a + 3] = (int32_t)W.sflag[a];
    float* f = sf + 9 * a;
    f[0] = hh.x; f[1] = hh.y; f[2] = hh.z;
    f[3] = ro.x; f[4] = ro.y; f[5] = ro.z;
    f[6] = rd.x; f[7] = rd.y; f[8] = rd.z;
  }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
static int persistent_blocks() { return 8 * num_sms(); }
static int traversal_limit(int32_t nf) { return 2 * (nf > 1 ? nf - 1 : 1) + 8; }

void launch_forward(const dt_scene& sc, const dt_views& vw, const dt_params& p, float* out, void* ws,
                    unsigned long long cap, cudaStream_t s) {
  WsView W = ws_view(ws, cap);
  cudaMemsetAsync(ws, 0, 1024, s);
  cudaMemsetAsync(out, 0, sizeof(float) * 3 * (size_t)vw.n_views * vw.width * vw.height, s);
  const uint64_t n0 = (uint64_t)vw.n_views * vw.width * vw.height * p.spp;
  int cb = (int)((n0 + 255) / 256);
  if (cb > 16 * num_sms()) cb = 16 * num_sms();
  {
    ProfScope ps("k_camera", s);
    k_camera<<<cb, 256, 0, s>>>(W, vw.d_cams, vw.n_views, vw.width, vw.height, p.spp, p.jitter, p.seed, cap,
                                p.max_depth);
  }
  BvhView B = bvh_view(sc.d_bvh, sc.nf);
  SceneDev S{sc.d_V, sc.d_F, sc.d_N, sc.d_ior, sc.d_sigma, sc.d_env, sc.env_w, sc.env_h};
  const uint32_t n_pix = (uint32_t)vw.n_views * vw.width * vw.height;
  for (int k = 0; k <= p.max_depth; ++k) {
    {
      ProfScope ps("k_trace", s);
      k_trace<<<persistent_blocks(), 256, 0, s>>>(W, B.nodes, B.tris, k, p.t_min, traversal_limit(sc.nf));
    }
    {
      ProfScope ps("k_shade", s);
      k_shade<<<persistent_blocks(), 256, 0, s>>>(W, S, k, p.max_depth, p.spp, n_pix, out);
    }
  }
}

void launch_dump(const void* ws, unsigned long long cap, int32_t* si, float* sf, unsigned long long n,
                 cudaStream_t s) {
  WsView W = ws_view(ws, cap);
  k_dump<<<4 * num_sms(), 256, 0, s>>>(W, si, sf, n);
}

void launch_closest_hit(const void* bvh, int32_t nf, const float* o, const float* d, const int32_t* src, int32_t n,
                        float tmin, int32_t* tri, float* tbb, cudaStream_t s) {
  BvhView B = bvh_view(bvh, nf);
  int b = (n + 127) / 128;
  if (b > 8 * num_sms()) b = 8 * num_sms();
  k_closest_hit_rays<<<b > 0 ? b : 1, 128, 0, s>>>(B.nodes, B.tris, o, d, src, n, tmin, traversal_limit(nf), tri,
                                                    tbb);
}

}  // namespace dt

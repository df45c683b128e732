// Backward of the recursive tracer: a reverse sweep over the tape, deepest
// level first.  For every segment s with radiance L_s it propagates
// gbar_s = dJ/dL_s = g_pixel * W_s / spp (W_s = forward throughput) through
// the operations of DiffTrans Sec. 3.3-3.4 at its hit:
//   L_s = A (R L_r + T L_t)   A = exp(-sigma t) inside (Eq. 11)
//   R, T = Fresnel (Eqs. 7-8); wr (Eq. 3); wt (Eqs. 4-6)
//   n = normalize(sum b_i N_i) (Eq. 12), N_v from Eq. 13
//   (t, b1, b2) from o + t d = v0 + b1 e1 + b2 e2 (hit point interpolated
//   from the vertex positions, Sec. 3.4 "Differentiable Mesh Intersection")
// and hands (L_s, dJ/do_s, dJ/dd_s) to its parent.  Vertex-position,
// vertex-normal, IoR and sigma gradients are accumulated atomically.
#include <cuda_runtime.h>
#include <stdint.h>

#include "dt_internal.cuh"
#include "dt_medium.cuh"
#include "dt_shade.cuh"

namespace dt {

extern dt_tuning g_tuning;

// An adjoint record (L, obar, dbar) of one segment: 9 floats in 36 bytes,
// as two float4 arrays (L.xyz obar.x | obar.yz dbar.xy) and one float array
// (dbar.z) of the level's length.
struct AdjRecords {
  float4* a;
  float4* b;
  float* c;
  __device__ __forceinline__ void load(uint32_t i, float3& L, float3& ob, float3& db) const {
    const float4 x = a[i], y = b[i];
    L = mk(x.x, x.y, x.z);
    ob = mk(x.w, y.x, y.y);
    db = mk(y.z, y.w, c[i]);
  }
  __device__ __forceinline__ void store(uint32_t i, float3 L, float3 ob, float3 db) const {
    a[i] = make_float4(L.x, L.y, L.z, ob.x);
    b[i] = make_float4(ob.y, ob.z, db.x, db.y);
    c[i] = db.z;
  }
};

// backward scratch: two level buffers of adjoint records and the dN/dV
// accumulators
struct BwsLayout {
  size_t off_buf[2][3], off_med, off_dN, total;
  BwsLayout(unsigned long long max_level, int32_t nv) {
    size_t o = 0;
    for (int k = 0; k < 2; ++k) {
      off_buf[k][0] = o;
      off_buf[k][1] = align_up(o + (size_t)max_level * sizeof(float4), 256);
      off_buf[k][2] = align_up(off_buf[k][1] + (size_t)max_level * sizeof(float4), 256);
      o = align_up(off_buf[k][2] + (size_t)max_level * sizeof(float), 256);
    }
    // per segment of the level being swept: (dJ/dS, t) of an interior
    // segment with an absorption grid, zeros otherwise
    off_med = o;
    o = align_up(o + (size_t)max_level * sizeof(float4), 256);
    off_dN = o;
    total = align_up(off_dN + (size_t)nv * 2 * sizeof(float4), 256);
  }
  AdjRecords records(void* base, int k) const {
    char* b = (char*)base;
    return AdjRecords{(float4*)(b + off_buf[k][0]), (float4*)(b + off_buf[k][1]), (float*)(b + off_buf[k][2])};
  }
};

// one 128-bit vector atomic per vertex (the accumulators are float4 per
// vertex, w unused)
__device__ __forceinline__ void atomic_add4(float4* p, float3 v) { atomicAdd(p, make_float4(v.x, v.y, v.z, 0.f)); }

// Per-scene gradient accumulators in the backward scratch: dN4 then dV4, nv
// float4 each; the entry's dN pointer holds their start.
__device__ __forceinline__ float4* acc_dN4(const SceneEntry& E) { return reinterpret_cast<float4*>(E.dN); }
__device__ __forceinline__ float4* acc_dV4(const SceneEntry& E) { return reinterpret_cast<float4*>(E.dN) + E.nv; }

// Per-block sums of the IoR and sigma gradients, one slot per scene; a thread
// adds its running sums when its scene changes and at the end.
struct SceneSums {
  float* s;  // shared [n_scenes][4]
  __device__ __forceinline__ void add(int scene, float ior, float3 sig) {
    if (scene < 0) return;
    if (ior != 0.f) atomicAdd(s + 4 * scene, ior);
    if (sig.x != 0.f) atomicAdd(s + 4 * scene + 1, sig.x);
    if (sig.y != 0.f) atomicAdd(s + 4 * scene + 2, sig.y);
    if (sig.z != 0.f) atomicAdd(s + 4 * scene + 3, sig.z);
  }
};

// out_next: (L, obar, dbar) of level k+1 indexed by position in that level;
// out_cur: the same for level k (not written for k = 0: camera rays have no
// parent); see AdjRecords.
// kBatch = false: one scene, whose entry E0 arrives as a kernel parameter;
// true: each segment looks its scene up.  kGrid: 1 = some scene has an
// absorption grid (dt_medium.cuh), whose optical depth interior segments add;
// 2 = some scene's is a hash texture.
constexpr int kAdjointMinBlocks = 3;  // CTAs of 256 per SM the register budget is sized for (80 registers)

// The attenuation A of an interior segment with an absorption grid, without
// marching its optical depth again: the forward gave each child the
// throughput W A F (F = R for the reflected child, T for the refracted one,
// rounded after each product), so A = W_child / (W F) to a few ulps.  The
// child with the larger factor is used (F >= 1/2; under TIR the reflected one
// with F = 1).  Where W F is not a normal float (a throughput driven to the
// subnormal range) the depth is marched as in the forward.
template <bool kHash>
__device__ __noinline__ float3 marched_absorption(const MediumView g, float3 o, float3 d, float t, float3 sigma) {
  return absorption_with_depth(sigma, t, medium_depth<kHash>(g, o, d, t));
}

template <bool kHash>
__device__ __forceinline__ float3 recovered_absorption(const WsView& W, const SceneEntry& E, const SceneEntry* Eg,
                                                       float4 rw, int32_t ch, uint32_t fl, bool tir,
                                                       const HitShade& h, float3 o, float3 d, float t,
                                                       float3 sigma) {
  const bool refl = tir || h.R >= 0.5f;
  const unsigned long long c = refl ? (unsigned long long)ch : (unsigned long long)ch + (fl >> kRefractShift);
  const float F = tir ? 1.0f : (refl ? h.R : h.T);
  const float3 den = mk(rw.x * F, rw.y * F, rw.z * F);
  if (c < W.cap && fminf(fminf(den.x, den.y), den.z) >= 1.17549435e-38f) {
    const float4 wc = W.ray_w[c];
    return mk(wc.x / den.x, wc.y / den.y, wc.z / den.z);
  }
  return marched_absorption<kHash>(medium_view(E, Eg), o, d, t, sigma);
}

template <bool kBatch, int kGrid>
__global__ void __launch_bounds__(256, kAdjointMinBlocks) k_adjoint(WsView W, int k, const AdjRecords out_next,
                                                                   const AdjRecords out_cur, const SceneEntry E0,
                                                                   float4* __restrict__ med_side) {
  extern __shared__ float sums_smem[];
  const WsHeader* H = W.hdr;
  const int n_scenes = kBatch ? W.th->n : 1;
  for (int i = threadIdx.x; i < 4 * n_scenes; i += blockDim.x) sums_smem[i] = 0.f;
  __syncthreads();
  SceneSums sums{sums_smem};
  const uint32_t n = level_size(H, k);
  const uint32_t start = H->level_start[k];
  const uint32_t next_start = H->level_start[k + 1];
  const uint32_t n_next = level_size(H, k + 1);
  int cur = -1;
  float acc_ior = 0.f;
  float3 acc_sig = mk(0.f, 0.f, 0.f);
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint32_t a = start + i;
    const float4 ro = W.ray_o[a], rd = W.ray_d[a], rw = W.ray_w[a];
    // the full tape keeps every hit record; a checkpointed one does not (see
    // the spawning branch below)
    const float4 hh = W.ring ? make_float4(0.f, 0.f, 0.f, 0.f) : W.hit[a];
    const uint32_t fl = W.sflag[a];
    const uint32_t sample = __float_as_uint(ro.w);
    const int sc = kBatch ? find_scene(W.th->starts, n_scenes, sample) : 0;
    const SceneEntry& E = kBatch ? W.ent[sc] : E0;
    if (sc != cur) {
      sums.add(cur, acc_ior, acc_sig);
      cur = sc;
      acc_ior = 0.f;
      acc_sig = mk(0.f, 0.f, 0.f);
    }
    const uint32_t pix = (sample - E.sample_start) / (uint32_t)E.spp;
    float3 L = mk(0.f, 0.f, 0.f), obar = L, dbar = L;
    float4 side = make_float4(0.f, 0.f, 0.f, 0.f);  // (dJ/dS, t) for the grid pass
    if (sample >= E.sample_start && pix < E.pix_count) {
      const float3 g = mk(__ldg(E.grad_out + 3 * (size_t)pix), __ldg(E.grad_out + 3 * (size_t)pix + 1),
                          __ldg(E.grad_out + 3 * (size_t)pix + 2));
      const float3 gbar = mul(g, mk(rw.x, rw.y, rw.z)) * (1.0f / (float)E.spp);
      const float3 o = xyz(ro), d = xyz(rd);
      const int32_t ch = W.child[a];
      if (fl & SF_MISS) {
        L = env_lookup(E.env, E.env_w, E.env_h, d);
        dbar = env_grad_dir(E.env, E.env_w, E.env_h, d, gbar);
      } else if (!(fl & (SF_DISCARDED | SF_BACKFACING)) && ch >= 0) {
        // checkpointed tape: the hit triangle is the source triangle its
        // children carry, and (t, b1, b2) come from intersecting it again
        // with the same arithmetic as the traversal's leaf test
        const int tri = W.ring ? __float_as_int(W.ray_w[ch].w) : __float_as_int(hh.w);
        const int i0 = __ldg(E.F + 3 * tri), i1 = __ldg(E.F + 3 * tri + 1), i2 = __ldg(E.F + 3 * tri + 2);
        const float3 v0 = load3(E.V + 3 * i0), v1 = load3(E.V + 3 * i1), v2 = load3(E.V + 3 * i2);
        float t = hh.x, b1 = hh.y, b2 = hh.z;
        if (W.ring) intersect_known(o, d, v0, v1 - v0, v2 - v0, t, b1, b2);
        const float b0 = 1.0f - b1 - b2;
        const float3 N0 = load3(E.N + 3 * i0), N1 = load3(E.N + 3 * i1), N2 = load3(E.N + 3 * i2);
        const float ior = __ldg(E.ior);
        const float3 sigma = mk(__ldg(E.sigma), __ldg(E.sigma + 1), __ldg(E.sigma + 2));
        const bool tir = (fl & SF_TIR) != 0;
        HitShade h;
        shade_hit(o, d, t, b1, b2, v0, v1, v2, N0, N1, N2, ior, sigma, h, tir ? 1 : 0);
        const bool med = kGrid && E.mu && !h.entering;
        if (med) h.A = recovered_absorption<kGrid == 2>(W, E, W.ent + sc, rw, ch, fl, tir, h, o, d, t, sigma);
        // children: reflected at ch, refracted at ch + (flags >> kRefractShift)
        float3 Lr = mk(0.f, 0.f, 0.f), orb = Lr, drb = Lr, Lt = Lr, otb = Lr, dtb = Lr;
        const uint32_t jr = (uint32_t)ch - next_start;
        const uint32_t jt = jr + (fl >> kRefractShift);
        if (jr < n_next) {
          out_next.load(jr, Lr, orb, drb);
        }
        if (!tir && jt < n_next) {
          out_next.load(jt, Lt, otb, dtb);
        }
        const float R = tir ? 1.0f : h.R, T = tir ? 0.0f : h.T;
        const float3 mix = Lr * R + Lt * T;
        L = mul(h.A, mix);
        // L = A (R Lr + T Lt)
        const float3 Abar = mul(gbar, mix);
        const float3 gA = mul(gbar, h.A);
        const float Rbar = dot(gA, Lr), Tbar = dot(gA, Lt);
        float tbar = 0.f;
        float3 sbar = mk(0.f, 0.f, 0.f);  // dJ/dS of the grid's optical depth
        if (!h.entering) {  // A_c = exp(-sigma_c t - S_c)
          const float3 aa = mul(Abar, h.A);
          acc_sig = acc_sig + aa * (-t);
          tbar -= dot(aa, sigma);
          if (med) {
            sbar = -aa;
            // tape_mode 2: dS/dt kept by the forward's medium pass (unless it did not march this segment)
            const bool kept = W.mom && !isnan(W.mom[kMomS * W.cap + a]);
            const float3 Sdt = kept ? mk(W.mom[(kMomDt + 0) * W.cap + a], W.mom[(kMomDt + 1) * W.cap + a],
                                         W.mom[(kMomDt + 2) * W.cap + a])
                                    : medium_depth_dt<kGrid == 2>(medium_view(E, W.ent + sc), o, d, t);
            tbar += dot(sbar, Sdt);
            side = make_float4(sbar.x, sbar.y, sbar.z, t);
          }
        }
        float cbar = 0.f, etabar = 0.f, eta1bar = 0.f, eta2bar = 0.f;
        float3 nsbar = mk(0.f, 0.f, 0.f), wibar = nsbar;
        if (!tir) {
          // R = (rs^2 + rp^2)/2, T = 1 - R
          const float Re = Rbar - Tbar;
          const float rsb = Re * h.rs, rpb = Re * h.rp;
          const float asb = rsb / h.bs_, bsb = -rsb * h.rs / h.bs_;
          const float apb = rpb / h.bp_, bpb = -rpb * h.rp / h.bp_;
          // rs = (eta1 c - eta2 cos_t) / (eta1 c + eta2 cos_t)
          eta1bar += (asb + bsb) * h.c;
          cbar += (asb + bsb) * h.eta1;
          eta2bar += (bsb - asb) * h.cos_t;
          float costb = (bsb - asb) * h.eta2;
          // rp = (eta1 cos_t - eta2 c) / (eta1 cos_t + eta2 c)
          eta1bar += (apb + bpb) * h.cos_t;
          costb += (apb + bpb) * h.eta1;
          eta2bar += (bpb - apb) * h.c;
          cbar += (bpb - apb) * h.eta2;
          // wt = (c ns - wi) / eta - cos_t ns
          const float3 wtb = dtb;
          const float3 q = h.ns * h.c - h.wi;
          wibar = wibar + wtb * (-1.0f / h.eta);
          cbar += dot(wtb, h.ns) / h.eta;
          nsbar = nsbar + wtb * (h.c / h.eta - h.cos_t);
          etabar -= dot(wtb, q) / (h.eta * h.eta);
          costb -= dot(wtb, h.ns);
          // cos_t = sqrt(kappa) / eta, kappa = eta^2 - 1 + c^2
          const float skb = costb / h.eta;
          etabar -= costb * h.cos_t / h.eta;
          const float kb = h.sk > 0.f ? skb * 0.5f / h.sk : 0.f;
          etabar += 2.0f * h.eta * kb;
          cbar += 2.0f * h.c * kb;
        }
        // wr = 2 c ns - wi
        cbar += 2.0f * dot(drb, h.ns);
        nsbar = nsbar + drb * (2.0f * h.c);
        wibar = wibar - drb;
        // eta = eta2 / eta1; the object's IoR is eta2 entering, eta1 leaving
        eta2bar += etabar / h.eta1;
        eta1bar -= etabar * h.eta / h.eta1;
        acc_ior += h.entering ? eta2bar : eta1bar;
        // c = wi . ns, wi = -d
        wibar = wibar + h.ns * cbar;
        nsbar = nsbar + h.wi * cbar;
        dbar = -wibar;
        // ns = +-n, n = m / |m|
        const float3 nbar = h.entering ? nsbar : -nsbar;
        const float3 mbar = (nbar - h.n * dot(h.n, nbar)) * (1.0f / h.lm);
        // m = b0 N0 + b1 N1 + b2 N2
        float4* dN4 = acc_dN4(E);
        atomic_add4(dN4 + i0, mbar * b0);
        atomic_add4(dN4 + i1, mbar * b1);
        atomic_add4(dN4 + i2, mbar * b2);
        const float b0b = dot(N0, mbar);
        const float b1b = dot(N1, mbar) - b0b;
        const float b2b = dot(N2, mbar) - b0b;
        // children start at x = o + t d
        const float3 xbar = orb + otb;
        obar = xbar;
        dbar = dbar + xbar * t;
        tbar += dot(xbar, d);
        // (t, b1, b2) solve o + t d - b0 v0 - b1 v1 - b2 v2 = 0; with
        // J = [d, -e1, -e2], lambda = -J^-T (tbar, b1bar, b2bar):
        // obar += lambda, dbar += t lambda, vibar -= bi lambda
        const float3 p = cross(d, h.e2);
        const float D3 = dot(d, h.ng);
        const float3 lam = D3 != 0.0f ? (h.ng * (-tbar) - p * b1b + cross(d, h.e1) * b2b) * (1.0f / D3)
                                      : mk(0.f, 0.f, 0.f);
        obar = obar + lam;
        dbar = dbar + lam * t;
        float4* dV4 = acc_dV4(E);
        atomic_add4(dV4 + i0, lam * (-b0));
        atomic_add4(dV4 + i1, lam * (-b1));
        atomic_add4(dV4 + i2, lam * (-b2));
      }
    }
    if (k > 0) {
      out_cur.store(i, L, obar, dbar);
    }
    if (kGrid) med_side[i] = side;
  }
  sums.add(cur, acc_ior, acc_sig);
  __syncthreads();
  for (int sc = threadIdx.x; sc < n_scenes; sc += blockDim.x) {
    const SceneEntry& E = kBatch ? W.ent[sc] : E0;
    if (sums_smem[4 * sc] != 0.f) atomicAdd(E.dior, sums_smem[4 * sc]);
    for (int c = 0; c < 3; ++c)
      if (sums_smem[4 * sc + 1 + c] != 0.f) atomicAdd(E.dsigma + c, sums_smem[4 * sc + 1 + c]);
  }
}

template <bool kBatch, bool kHash>
__device__ __forceinline__ void medium_adjoint_one(const WsView& W, int k, const AdjRecords& out_cur,
                                                   const float4* __restrict__ med_side, const SceneEntry& E0,
                                                   uint32_t start, int n_scenes, uint32_t i) {
  const float4 sv = med_side[i];
  const uint32_t a = start + i;
  const float4 ro = W.ray_o[a], rd = W.ray_d[a];
  const int sc = kBatch ? find_scene(W.th->starts, n_scenes, __float_as_uint(ro.w)) : 0;
  const SceneEntry& E = kBatch ? W.ent[sc] : E0;
  if (!E.mu) return;
  float3 ob = mk(0.f, 0.f, 0.f), db = ob;
  const float3 sbar = mk(sv.x, sv.y, sv.z);
  if (W.mom && !isnan(W.mom[kMomS * W.cap + a])) {
    // tape_mode 2: the samples' motion from the forward's moments, so only
    // the scatter into the table marches the segment
    const float* M = W.mom + a;
    const unsigned long long c = W.cap;
    ob = mk(sbar.x * M[(kMomDo + 0) * c] + sbar.y * M[(kMomDo + 3) * c] + sbar.z * M[(kMomDo + 6) * c],
            sbar.x * M[(kMomDo + 1) * c] + sbar.y * M[(kMomDo + 4) * c] + sbar.z * M[(kMomDo + 7) * c],
            sbar.x * M[(kMomDo + 2) * c] + sbar.y * M[(kMomDo + 5) * c] + sbar.z * M[(kMomDo + 8) * c]);
    db = mk(sbar.x * M[(kMomDd + 0) * c] + sbar.y * M[(kMomDd + 3) * c] + sbar.z * M[(kMomDd + 6) * c],
            sbar.x * M[(kMomDd + 1) * c] + sbar.y * M[(kMomDd + 4) * c] + sbar.z * M[(kMomDd + 7) * c],
            sbar.x * M[(kMomDd + 2) * c] + sbar.y * M[(kMomDd + 5) * c] + sbar.z * M[(kMomDd + 8) * c]);
    if (E.dmu) medium_scatter<kHash>(medium_view(E, W.ent + sc), E.dmu, xyz(ro), xyz(rd), sv.w, sbar);
  } else {
    medium_backward<kHash>(medium_view(E, W.ent + sc), E.dmu, xyz(ro), xyz(rd), sv.w, sbar, ob, db);
  }
  if (k > 0) {  // camera rays have no parent to hand (obar, dbar) to
    float3 L, o0, d0;
    out_cur.load(i, L, o0, d0);
    out_cur.store(i, L, o0 + ob, d0 + db);
  }
}

// The absorption grid's share of the adjoint of level k, after k_adjoint:
// for each interior segment with a grid (side = (dJ/dS, t), t > 0) the
// samples of its optical depth move with the segment's o and d at fixed t,
// which adds to its adjoint record (read by the parent level next), and
// dJ/dS goes to the grid's nodes.  A pass of its own, so the march and the
// node atomics run at the occupancy of a small kernel.  kHash: some scene's
// grid is a hash texture.  About half of a level's segments run inside the
// object; a warp gathers the positions that do into a queue in shared
// memory and marches them 32 at a time, so that its lanes are not left idle
// beside the segments that need no march.
constexpr int kMedAdjWarps = 8;
template <bool kBatch, bool kHash>
__global__ void __launch_bounds__(32 * kMedAdjWarps, 3) k_medium_adjoint(WsView W, int k, const AdjRecords out_cur,
                                                                       const float4* __restrict__ med_side,
                                                                       const SceneEntry E0) {
  __shared__ uint32_t s_queue[kMedAdjWarps][64];
  const WsHeader* H = W.hdr;
  const int n_scenes = kBatch ? W.th->n : 1;
  const uint32_t n = level_size(H, k);
  const uint32_t start = H->level_start[k];
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t* q = s_queue[wid];
  const uint32_t warps = gridDim.x * kMedAdjWarps;
  uint32_t cnt = 0;  // queued positions (warp-uniform, < 64)
  for (uint32_t base = (blockIdx.x * kMedAdjWarps + wid) * 32u;; base += warps * 32u) {
    const bool more = base < n;
    if (more) {
      const uint32_t i = base + lane;
      bool v = false;
      if (i < n) {
        const float4 sv = med_side[i];
        v = sv.w > 0.f && !(sv.x == 0.f && sv.y == 0.f && sv.z == 0.f);  // a grid, and a gradient
      }
      const unsigned b = __ballot_sync(kFull, v);
      if (v) q[cnt + __popc(b & ((1u << lane) - 1u))] = i;
      cnt += (uint32_t)__popc(b);
      __syncwarp();
    }
    while (cnt >= 32u || (!more && cnt > 0u)) {
      const uint32_t take = cnt < 32u ? cnt : 32u;
      if (lane < take) medium_adjoint_one<kBatch, kHash>(W, k, out_cur, med_side, E0, start, n_scenes, q[lane]);
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
}

// Gradient of the environment texels (Sec. 3.4 step 3 read with a bilinear
// lookup, linear in the texels): every segment that missed adds gbar =
// g_pixel W / spp times its four bilinear weights to four texels.  It needs
// no adjoint of other segments, so one pass covers every level of the tape.
// kShared: one scene whose environment fits a CTA's shared memory; its texels
// are summed there first and added to the output with one atomic per texel
// per CTA (the bench's 64x32 environment takes tens of millions of misses
// per step, which global atomics on 2048 texels would serialise).  Each
// thread takes a contiguous chunk of the tape, so a warp's lanes read rays
// far apart (other pixels, other directions) and rarely add to the same
// texel in one instruction, as arena neighbours (coherent rays) would.
constexpr int kEnvSharedTexels = 4096;  // 48 KB of float sums

template <bool kBatch, bool kShared>
__global__ void __launch_bounds__(256) k_env_adjoint(WsView W, const SceneEntry E0) {
  extern __shared__ float env_acc[];
  const WsHeader* H = W.hdr;
  const int n_scenes = kBatch ? W.th->n : 1;
  const int nl = (int)H->n_levels;
  const unsigned long long total = nl > 0 ? H->level_start[nl] : 0ull;
  const unsigned long long lim = total < W.cap ? total : W.cap;
  const int ntex3 = kShared ? 3 * E0.env_w * E0.env_h : 0;
  if (kShared) {
    for (int i = threadIdx.x; i < ntex3; i += blockDim.x) env_acc[i] = 0.f;
    __syncthreads();
  }
  const unsigned long long nthreads = (unsigned long long)gridDim.x * blockDim.x;
  const unsigned long long chunk = (lim + nthreads - 1) / nthreads;
  const unsigned long long a0 = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) * chunk;
  const unsigned long long a1 = a0 + chunk < lim ? a0 + chunk : lim;
  constexpr int kU = 4;  // segments in flight per thread
  for (unsigned long long a = a0; a < a1; a += kU) {
    bool miss[kU];
    float4 ro[kU], rd[kU], rw[kU];
#pragma unroll
    for (int j = 0; j < kU; ++j) miss[j] = a + j < a1 && (W.sflag[a + j] & SF_MISS);
#pragma unroll
    for (int j = 0; j < kU; ++j)
      if (miss[j]) {
        ro[j] = W.ray_o[a + j];
        rd[j] = W.ray_d[a + j];
        rw[j] = W.ray_w[a + j];
      }
#pragma unroll
    for (int j = 0; j < kU; ++j) {
      if (!miss[j]) continue;
      const uint32_t sample = __float_as_uint(ro[j].w);
      const SceneEntry& E = kBatch ? W.ent[find_scene(W.th->starts, n_scenes, sample)] : E0;
      if (!E.denv) continue;
      const uint32_t pix = (sample - E.sample_start) / (uint32_t)E.spp;
      if (sample < E.sample_start || pix >= E.pix_count) continue;  // a dead record
      const float3 g = mk(__ldg(E.grad_out + 3 * (size_t)pix), __ldg(E.grad_out + 3 * (size_t)pix + 1),
                          __ldg(E.grad_out + 3 * (size_t)pix + 2));
      const float3 gbar = mul(g, mk(rw[j].x, rw[j].y, rw[j].z)) * (1.0f / (float)E.spp);
      const EnvSample es = env_coords(xyz(rd[j]), E.env_w, E.env_h);
      const int tex[4] = {es.y0 * E.env_w + es.x0, es.y0 * E.env_w + es.x1, es.y1 * E.env_w + es.x0,
                          es.y1 * E.env_w + es.x1};
      const float wt[4] = {(1.0f - es.ax) * (1.0f - es.ay), es.ax * (1.0f - es.ay), (1.0f - es.ax) * es.ay,
                           es.ax * es.ay};
      float* dst = kShared ? env_acc : E.denv;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        atomicAdd(dst + 3 * tex[q], gbar.x * wt[q]);
        atomicAdd(dst + 3 * tex[q] + 1, gbar.y * wt[q]);
        atomicAdd(dst + 3 * tex[q] + 2, gbar.z * wt[q]);
      }
    }
  }
  if (kShared) {
    __syncthreads();
    for (int i = threadIdx.x; i < ntex3; i += blockDim.x)
      if (env_acc[i] != 0.f) atomicAdd(E0.denv + i, env_acc[i]);
  }
}

// zero every scene's accumulators, dIoR, dsigma and absorption-grid
// gradient (blockIdx.y = scene)
__global__ void k_zero_grads(const SceneEntry* __restrict__ ent) {
  const SceneEntry& E = ent[blockIdx.y];
  const size_t n = 2 * (size_t)E.nv;
  float4* acc = acc_dN4(E);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    acc[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (E.mu && E.dmu) {
    const size_t nn = E.gentries;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nn; i += (size_t)gridDim.x * blockDim.x)
      E.dmu[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  if (E.denv) {
    const size_t ne = 3 * (size_t)E.env_w * E.env_h;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < ne; i += (size_t)gridDim.x * blockDim.x)
      E.denv[i] = 0.f;
  }
  if (blockIdx.x == 0 && threadIdx.x < 4) {
    if (threadIdx.x == 0) E.dior[0] = 0.f;
    else E.dsigma[threadIdx.x - 1] = 0.f;
  }
}

// Eq. 13 backward for every scene (blockIdx.y = scene): dN -> dV, on the
// float4 accumulators (the same arithmetic as face_normal_backward_one)
__global__ void k_face_normals_backward_table(const SceneEntry* __restrict__ ent) {
  const SceneEntry& E = ent[blockIdx.y];
  const float4* dN4 = acc_dN4(E);
  float4* dV4 = acc_dV4(E);
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < E.nf; f += gridDim.x * blockDim.x) {
    const int i0 = E.F[3 * f], i1 = E.F[3 * f + 1], i2 = E.F[3 * f + 2];
    const float3 v0 = load3(E.V + 3 * i0), v1 = load3(E.V + 3 * i1), v2 = load3(E.V + 3 * i2);
    const float3 e1 = v1 - v0, e2 = v2 - v0;
    const float3 c = cross_rn(e1, e2);
    const float lc = len(c);
    if (!(lc > 0.0f)) continue;  // a zero-area face added nothing to the normals
    const float3 u = mk(c.x / lc, c.y / lc, c.z / lc);
    const float3 du = (xyz(dN4[i0]) + xyz(dN4[i1]) + xyz(dN4[i2])) * (1.0f / 3.0f);
    const float3 dc = (du - u * dot(u, du)) * (1.0f / lc);
    const float3 de1 = cross(e2, dc), de2 = cross(dc, e1);
    atomic_add4(dV4 + i0, -(de1 + de2));
    atomic_add4(dV4 + i1, de1);
    atomic_add4(dV4 + i2, de2);
  }
}

// the caller's dV [nv][3] from the accumulator (blockIdx.y = scene)
__global__ void k_finish_grads_table(const SceneEntry* __restrict__ ent) {
  const SceneEntry& E = ent[blockIdx.y];
  const float4* dV4 = acc_dV4(E);
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < E.nv; v += gridDim.x * blockDim.x) {
    const float4 g = dV4[v];
    E.dV[3 * v] = g.x;
    E.dV[3 * v + 1] = g.y;
    E.dV[3 * v + 2] = g.z;
  }
}

// L2 seed: grad = 2 scale (img - target); loss = scale sum (img - target)^2
__global__ void k_l2_loss_grad(const float* __restrict__ img, const float* __restrict__ target, int64_t n,
                               float scale, float* __restrict__ grad, float* __restrict__ loss) {
  float acc = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float r = img[i] - target[i];
    grad[i] = 2.0f * scale * r;
    acc += r * r;
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0 && acc != 0.f) atomicAdd(loss, acc * scale);
}

// Eqs. 14-15 per pixel and their gradient; loss[0..2] gather (total,
// L_color, L_tone) with one atomic each per warp.
__global__ void k_paper_loss_grad(const float* __restrict__ img, const float* __restrict__ target, int64_t n,
                                  float inv_n, float lc, float lt, float* __restrict__ grad,
                                  float* __restrict__ loss) {
  float acc_c = 0.f, acc_t = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float3 ch = load3(img + 3 * i), c = load3(target + 3 * i);
    const float3 r = mul(ch - c, c);
    acc_c += dot(r, r);
    float3 g = mul(r, c) * (2.0f * inv_n * lc);
    const float mean = (c.x + c.y + c.z) * (1.0f / 3.0f);
    const float var = ((c.x - mean) * (c.x - mean) + (c.y - mean) * (c.y - mean) + (c.z - mean) * (c.z - mean)) *
                      (1.0f / 3.0f);
    const float nh = len(ch), nc = len(c);
    if (nh > 0.0f && nc > 0.0f) {
      const float s = dot(ch, c) / (nh * nc);
      const float3 ds = c * (1.0f / (nh * nc)) - ch * (s / (nh * nh));
      g = g + ds * (-2.0f * (1.0f - s) * inv_n * lt);
      acc_t += (1.0f - s) * (1.0f - s) - var;
    } else {
      acc_t += 1.0f - var;
    }
    grad[3 * i] = g.x;
    grad[3 * i + 1] = g.y;
    grad[3 * i + 2] = g.z;
  }
  acc_c = warp_sum(acc_c) * inv_n;
  acc_t = warp_sum(acc_t) * inv_n;
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(loss, lc * acc_c + lt * acc_t);
    atomicAdd(loss + 1, acc_c);
    atomicAdd(loss + 2, acc_t);
  }
}

void launch_paper_loss_grad(const float* img, const float* target, int64_t n, float lc, float lt, float* grad,
                            float* loss, cudaStream_t s) {
  cudaMemsetAsync(loss, 0, 3 * sizeof(float), s);
  if (n == 0) return;
  int64_t b = (n + 255) / 256;
  if (b > 8 * num_sms()) b = 8 * num_sms();
  ProfScope ps("k_paper_loss_grad", s);
  k_paper_loss_grad<<<(int)b, 256, 0, s>>>(img, target, n, 1.0f / (float)n, lc, lt, grad, loss);
}

void launch_l2_loss_grad(const float* img, const float* target, int64_t n, float scale, float* grad, float* loss,
                         cudaStream_t s) {
  cudaMemsetAsync(loss, 0, sizeof(float), s);
  if (n == 0) return;
  int64_t b = (n + 255) / 256;
  if (b > 8 * num_sms()) b = 8 * num_sms();
  ProfScope ps("k_l2_loss_grad", s);
  k_l2_loss_grad<<<(int)b, 256, 0, s>>>(img, target, n, scale, grad, loss);
}

void launch_write_table(const WsView& W, const TableHeader& th, const SceneEntry* entries, int n, cudaStream_t s);

// Backward of a table of scenes over the tape in ws: rewrites the table with
// the gradient pointers, zeroes the gradients, sweeps k = D..0, then the
// vertex-normal adjoint of every scene.
void launch_backward_table(const TableHeader& th, const SceneEntry* entries, const void* ws, unsigned long long cap,
                           unsigned long long ring, bool mom, void* bws, unsigned long long max_level, cudaStream_t s) {
  WsView W = ws_view(ws, cap, ring, mom);
  BwsLayout L(max_level, 0);
  const AdjRecords buf[2] = {L.records(bws, 0), L.records(bws, 1)};
  const int n = th.n;
  launch_write_table(W, th, entries, n, s);
  int max_nv = 1, max_nf = 1;
  for (int i = 0; i < n; ++i) {
    if (entries[i].nv > max_nv) max_nv = entries[i].nv;
    if (entries[i].nf > max_nf) max_nf = entries[i].nf;
  }
  const int cap_blocks = 4 * num_sms();
  int zb = (2 * max_nv + 255) / 256;
  if (zb > cap_blocks) zb = cap_blocks;
  {
    ProfScope ps("k_zero_grads", s);
    k_zero_grads<<<dim3(zb, n), 256, 0, s>>>(W.ent);
  }
  const int blocks = kAdjointMinBlocks * num_sms();  // one wave of the resident CTAs
  const size_t smem = sizeof(float) * 4 * (size_t)n;
  float4* side = reinterpret_cast<float4*>((char*)bws + L.off_med);
  for (int k = th.max_depth; k >= 0; --k) {
    const AdjRecords nx = buf[(k + 1) & 1], cu = buf[k & 1];
    {
      ProfScope ps("k_adjoint", s);
      if (th.any_medium == 2) {
        if (n > 1) k_adjoint<true, 2><<<blocks, 256, smem, s>>>(W, k, nx, cu, entries[0], side);
        else k_adjoint<false, 2><<<blocks, 256, smem, s>>>(W, k, nx, cu, entries[0], side);
      } else if (th.any_medium) {
        if (n > 1) k_adjoint<true, 1><<<blocks, 256, smem, s>>>(W, k, nx, cu, entries[0], side);
        else k_adjoint<false, 1><<<blocks, 256, smem, s>>>(W, k, nx, cu, entries[0], side);
      } else {
        if (n > 1) k_adjoint<true, 0><<<blocks, 256, smem, s>>>(W, k, nx, cu, entries[0], side);
        else k_adjoint<false, 0><<<blocks, 256, smem, s>>>(W, k, nx, cu, entries[0], side);
      }
    }
    if (th.any_medium) {
      ProfScope ps("k_medium_adjoint", s);
      const int mb = 8 * num_sms();
      if (th.any_medium == 2) {
        if (n > 1) k_medium_adjoint<true, true><<<mb, 256, 0, s>>>(W, k, cu, side, entries[0]);
        else k_medium_adjoint<false, true><<<mb, 256, 0, s>>>(W, k, cu, side, entries[0]);
      } else {
        if (n > 1) k_medium_adjoint<true, false><<<mb, 256, 0, s>>>(W, k, cu, side, entries[0]);
        else k_medium_adjoint<false, false><<<mb, 256, 0, s>>>(W, k, cu, side, entries[0]);
      }
    }
  }
  if (th.any_env_grad) {
    ProfScope ps("k_env_adjoint", s);
    const SceneEntry& E0 = entries[0];
    const int tex = E0.env_w * E0.env_h;
    if (n > 1) k_env_adjoint<true, false><<<4 * num_sms(), 256, 0, s>>>(W, E0);
    else if (tex <= kEnvSharedTexels)
      k_env_adjoint<false, true><<<4 * num_sms(), 256, 3 * sizeof(float) * (size_t)tex, s>>>(W, E0);
    else k_env_adjoint<false, false><<<4 * num_sms(), 256, 0, s>>>(W, E0);
  }
  int fb = (max_nf + 255) / 256;
  if (fb > cap_blocks) fb = cap_blocks;
  ProfScope ps("k_face_normals_backward", s);
  k_face_normals_backward_table<<<dim3(fb, n), 256, 0, s>>>(W.ent);
  int vb = (max_nv + 255) / 256;
  if (vb > cap_blocks) vb = cap_blocks;
  k_finish_grads_table<<<dim3(vb, n), 256, 0, s>>>(W.ent);
}

// The backward scratch of a table: the two level buffers, then every
// scene's dN and dV accumulators (float4 per vertex each).  assign_dN
// points each entry's dN at its pair.
size_t backward_ws_bytes_table(unsigned long long max_level, const SceneEntry* entries, int n) {
  BwsLayout L(max_level, 0);
  size_t o = L.off_dN;
  for (int i = 0; i < n; ++i) o = align_up(o + (size_t)entries[i].nv * 2 * sizeof(float4), 256);
  return o;
}

void assign_dN(SceneEntry* entries, int n, void* bws, unsigned long long max_level) {
  BwsLayout L(max_level, 0);
  size_t o = L.off_dN;
  for (int i = 0; i < n; ++i) {
    entries[i].dN = (float*)((char*)bws + o);
    o = align_up(o + (size_t)entries[i].nv * 2 * sizeof(float4), 256);
  }
}

}  // namespace dt

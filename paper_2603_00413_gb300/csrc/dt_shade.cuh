// Per-hit optics of DiffTrans Sec. 3.3-3.4 in FP32, written once and used by
// the forward shading kernel and by the adjoint kernel (which recomputes the
// forward quantities it differentiates).
#pragma once

#include "dt_internal.cuh"

namespace dt {

constexpr float kPi = 3.14159265358979323846f;

// Equirectangular environment, y up: phi = atan2(dz, dx) in [0, 2pi),
// theta = acos(dy); texel coordinates u = phi/(2pi) W - 1/2,
// v = theta/pi H - 1/2; bilinear, wrapping in u, clamping in v.
struct EnvSample {
  int x0, x1, y0, y1;
  float ax, ay;
  float u, v;
  float phi_dx, phi_dz;  // d phi / d(dx, dz)
  float theta_dy;        // d theta / d dy (0 where dy is clamped)
};

__device__ __forceinline__ EnvSample env_coords(float3 d, int W, int H) {
  EnvSample s;
  float phi = atan2f(d.z, d.x);
  if (phi < 0.0f) phi = phi + 2.0f * kPi;
  const float cy = fminf(fmaxf(d.y, -1.0f), 1.0f);
  const float theta = acosf(cy);
  s.u = phi / (2.0f * kPi) * (float)W - 0.5f;
  s.v = theta / kPi * (float)H - 0.5f;
  const float fu = floorf(s.u), fv = floorf(s.v);
  s.ax = s.u - fu;
  s.ay = s.v - fv;
  int x0 = (int)fu, y0 = (int)fv;
  int x1 = x0 + 1, y1 = y0 + 1;
  x0 = ((x0 % W) + W) % W;
  x1 = ((x1 % W) + W) % W;
  y0 = min(max(y0, 0), H - 1);
  y1 = min(max(y1, 0), H - 1);
  s.x0 = x0; s.x1 = x1; s.y0 = y0; s.y1 = y1;
  const float r2 = d.x * d.x + d.z * d.z;
  s.phi_dx = r2 > 1e-30f ? -d.z / r2 : 0.0f;  // azimuth undefined on the pole axis
  s.phi_dz = r2 > 1e-30f ? d.x / r2 : 0.0f;
  s.theta_dy = (d.y > -1.0f && d.y < 1.0f) ? -1.0f / sqrtf(1.0f - d.y * d.y) : 0.0f;
  return s;
}

__device__ __forceinline__ float3 env_tex(const float* env, int W, int y, int x) {
  const float* p = env + 3 * ((size_t)y * W + x);
  return mk(__ldg(p), __ldg(p + 1), __ldg(p + 2));
}

__device__ __forceinline__ float3 env_eval(const float* env, int W, const EnvSample& s) {
  const float3 t00 = env_tex(env, W, s.y0, s.x0), t10 = env_tex(env, W, s.y0, s.x1);
  const float3 t01 = env_tex(env, W, s.y1, s.x0), t11 = env_tex(env, W, s.y1, s.x1);
  const float w00 = (1.0f - s.ax) * (1.0f - s.ay), w10 = s.ax * (1.0f - s.ay);
  const float w01 = (1.0f - s.ax) * s.ay, w11 = s.ax * s.ay;
  return t00 * w00 + t10 * w10 + t01 * w01 + t11 * w11;
}

__device__ __forceinline__ float3 env_lookup(const float* env, int W, int H, float3 d) {
  return env_eval(env, W, env_coords(d, W, H));
}

// Gradient of g . E(d) with respect to d (g per channel).
__device__ __forceinline__ float3 env_grad_dir(const float* env, int W, int H, float3 d, float3 g) {
  const EnvSample s = env_coords(d, W, H);
  const float3 t00 = env_tex(env, W, s.y0, s.x0), t10 = env_tex(env, W, s.y0, s.x1);
  const float3 t01 = env_tex(env, W, s.y1, s.x0), t11 = env_tex(env, W, s.y1, s.x1);
  const float3 dEdax = (t10 - t00) * (1.0f - s.ay) + (t11 - t01) * s.ay;
  const float3 dEday = (t01 - t00) * (1.0f - s.ax) + (t11 - t10) * s.ax;
  const float gu = dot(g, dEdax) * ((float)W / (2.0f * kPi));  // d/dphi
  const float gv = dot(g, dEday) * ((float)H / kPi);           // d/dtheta
  return mk(gu * s.phi_dx, gv * s.theta_dy, gu * s.phi_dz);
}

// Forward quantities at one hit (everything the adjoint differentiates).
struct HitShade {
  float3 e1, e2, ng;  // triangle edges and geometric normal e1 x e2
  float3 x;           // hit point o + t d
  float3 m;           // un-normalised interpolated normal (Eq. 12)
  float lm;           // |m|
  float3 n, ns;       // unit normal, turned toward the incoming side
  float3 wi;          // -d
  float c;            // cos(theta_i) = wi . ns
  float eta1, eta2, eta;
  float3 wr, wt;      // reflected (Eq. 3) and refracted (Eqs. 4-6) directions
  float kappa, sk, cos_t;
  float as_, bs_, rs, ap_, bp_, rp;
  float R, T;         // Eqs. 7-8
  float3 A;           // absorption over this segment (Eq. 11)
  bool entering, backfacing, tir;
};

// t, b1, b2: the stored intersection; N0..N2 vertex normals; ior, sigma.
// tir_mode < 0 decides total internal reflection from kappa; 0 or 1 imposes
// the decision the forward pass stored (a recomputation in another kernel may
// round kappa to the other side of 0; kappa is then clamped at 0).
__device__ __forceinline__ void shade_hit(float3 o, float3 d, float t, float b1, float b2, float3 v0, float3 v1,
                                          float3 v2, float3 N0, float3 N1, float3 N2, float ior, float3 sigma,
                                          HitShade& h, int tir_mode = -1) {
  h.e1 = v1 - v0;
  h.e2 = v2 - v0;
  h.ng = cross(h.e1, h.e2);
  h.entering = dot(d, h.ng) < 0.0f;  // Sec. 3.4 step 2: from outside or inside
  const float b0 = 1.0f - b1 - b2;
  h.x = o + d * t;
  h.m = N0 * b0 + N1 * b1 + N2 * b2;
  h.lm = len(h.m);
  h.n = mk(h.m.x / h.lm, h.m.y / h.lm, h.m.z / h.lm);
  h.ns = h.entering ? h.n : -h.n;
  h.wi = -d;
  h.c = dot(h.wi, h.ns);
  h.backfacing = !(h.c > 0.0f);
  h.eta1 = h.entering ? 1.0f : ior;
  h.eta2 = h.entering ? ior : 1.0f;
  h.eta = h.eta2 / h.eta1;
  h.wr = (2.0f * h.c) * h.ns - h.wi;                   // Eq. 3
  h.kappa = h.eta * h.eta - (1.0f - h.c * h.c);       // eta^2 - sin^2(theta_i)
  h.tir = tir_mode < 0 ? h.kappa < 0.0f : tir_mode != 0;
  if (!h.tir && h.kappa < 0.0f) h.kappa = 0.0f;
  if (h.tir) {
    h.sk = 0.f; h.cos_t = 0.f; h.wt = mk(0.f, 0.f, 0.f);
    h.as_ = h.bs_ = h.rs = h.ap_ = h.bp_ = h.rp = 0.f;
    h.R = 1.0f; h.T = 0.0f;
  } else {
    h.sk = sqrtf(h.kappa);
    h.cos_t = h.sk / h.eta;
    const float3 w_par = (-h.cos_t) * h.ns;            // Eq. 5
    const float3 w_perp = (h.wi - h.c * h.ns) * (-1.0f / h.eta);  // Eq. 6
    h.wt = w_perp + w_par;                             // Eq. 4
    h.as_ = h.eta1 * h.c - h.eta2 * h.cos_t;
    h.bs_ = h.eta1 * h.c + h.eta2 * h.cos_t;
    h.rs = h.as_ / h.bs_;
    h.ap_ = h.eta1 * h.cos_t - h.eta2 * h.c;
    h.bp_ = h.eta1 * h.cos_t + h.eta2 * h.c;
    h.rp = h.ap_ / h.bp_;
    h.R = 0.5f * (h.rs * h.rs + h.rp * h.rp);          // Eq. 7
    h.T = 1.0f - h.R;                                  // Eq. 8
  }
  if (h.entering) {
    h.A = mk(1.0f, 1.0f, 1.0f);
  } else {                                             // Sec. 3.4 step 5
    h.A = mk(expf(-sigma.x * t), expf(-sigma.y * t), expf(-sigma.z * t));
  }
}

// Absorption of an interior segment whose optical depth sigma t gains the
// depth S of an absorption grid (Eq. 11 with a spatially varying rate).
__device__ __forceinline__ float3 absorption_with_depth(float3 sigma, float t, float3 S) {
  return mk(expf(-(sigma.x * t + S.x)), expf(-(sigma.y * t + S.y)), expf(-(sigma.z * t + S.z)));
}

// Moller-Trumbore of one triangle (v0, e1 = v1 - v0, e2 = v2 - v0): (t, b1,
// b2) with o + t d = v0 + b1 e1 + b2 e2; false when d is parallel to the
// plane.  The traversal's leaf test evaluates the same expressions in the
// same order on the same inputs (e1, e2 as the refit stores them), so the
// checkpointed backward recovers the forward's hit.
__device__ __forceinline__ bool intersect_known(float3 o, float3 d, float3 v0, float3 e1, float3 e2, float& t,
                                                float& b1, float& b2) {
  const float3 p = cross(d, e2);
  const float det = dot(e1, p);
  if (det == 0.0f) return false;
  const float inv = 1.0f / det;
  const float3 s = o - v0;
  b1 = dot(s, p) * inv;
  const float3 q = cross(s, e1);
  b2 = dot(d, q) * inv;
  t = dot(e2, q) * inv;
  return true;
}

// Backward of Eq. 13 for face f.  Its unit normal u = c/|c|, c = e1 x e2,
// feeds (1/3) u to each of its vertices, so du = (1/3)(dN_v0 + dN_v1 +
// dN_v2); dc = (du - u (u.du)) / |c|; c = e1 x e2 gives de1 = e2 x dc,
// de2 = dc x e1; then dv1 += de1, dv2 += de2, dv0 -= de1 + de2 (atomics).
__device__ __forceinline__ void face_normal_backward_one(const float* __restrict__ V, const int32_t* __restrict__ F,
                                                         int f, const float* __restrict__ dN, float* __restrict__ dV) {
  const int i0 = F[3 * f], i1 = F[3 * f + 1], i2 = F[3 * f + 2];
  const float3 v0 = load3(V + 3 * i0), v1 = load3(V + 3 * i1), v2 = load3(V + 3 * i2);
  const float3 e1 = v1 - v0, e2 = v2 - v0;
  const float3 c = cross_rn(e1, e2);
  const float lc = len(c);
  if (!(lc > 0.0f)) return;  // a zero-area face added nothing to the normals
  const float3 u = mk(c.x / lc, c.y / lc, c.z / lc);
  const float3 du = (load3(dN + 3 * i0) + load3(dN + 3 * i1) + load3(dN + 3 * i2)) * (1.0f / 3.0f);
  const float3 dc = (du - u * dot(u, du)) * (1.0f / lc);
  const float3 de1 = cross(e2, dc), de2 = cross(dc, e1);
  const float3 dv0 = -(de1 + de2);
  atomicAdd(dV + 3 * i0 + 0, dv0.x); atomicAdd(dV + 3 * i0 + 1, dv0.y); atomicAdd(dV + 3 * i0 + 2, dv0.z);
  atomicAdd(dV + 3 * i1 + 0, de1.x); atomicAdd(dV + 3 * i1 + 1, de1.y); atomicAdd(dV + 3 * i1 + 2, de1.z);
  atomicAdd(dV + 3 * i2 + 0, de2.x); atomicAdd(dV + 3 * i2 + 1, de2.y); atomicAdd(dV + 3 * i2 + 2, de2.z);
}

}  // namespace dt

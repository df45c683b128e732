// Spatially varying absorption (DiffTrans Eq. 11 with mu_t(x) = sigma +
// G(x)): G is a dense grid of per-channel rates at the nodes of an
// nx x ny x nz lattice over a box, read with trilinear interpolation at
// positions clamped to the box.  Over an interior segment o + s d, s in
// [0, t], the optical depth gains the sum of Eq. 11 over steps of length h
// from the segment's start: m = floor(t / h) full steps (at most
// kMaxMediumSteps) and a last one of length r = t - m h, each sampled at its
// midpoint and weighted by its length.  The sum is continuous in t (the
// partial step grows into the next full one), so only the partial step
// depends on t:
//   dS/dt = G(x_m) + (r / 2) dG/dx(x_m) d,
// and at fixed t every sample moves with o and d:
//   dS/do = sum_i w_i dG/dx(x_i),  dS/dd = sum_i w_i s_i dG/dx(x_i).
// The forward shading pass and the adjoint evaluate S and dS/dt; a separate
// pass over the interior segments of each level adds the o and d terms to
// their adjoint records and scatters dJ/dS w_i into the eight nodes of each
// sample's cell.
#pragma once

#include "dt_internal.cuh"

namespace dt {

constexpr int kMaxMediumSteps = 8192;

struct MediumView {
  const float4* mu;
  int nx, ny, nz;
  float3 lo, scale;
  float step;
};

__device__ __forceinline__ MediumView medium_view(const SceneEntry& E) {
  return MediumView{E.mu, E.gnx, E.gny, E.gnz, mk(E.glo_x, E.glo_y, E.glo_z),
                    mk(E.gscale_x, E.gscale_y, E.gscale_z), E.gstep};
}

// Cell of x: per axis u = (x - lo) scale clamped to [0, n - 1], cell index
// min(floor(u), n - 2) and fraction u - index; `free` = the axis was not
// clamped (a clamped coordinate is constant, so it has no derivative).
struct GridCell {
  size_t base;             // node index of the cell's (0, 0, 0) corner
  int sx, sy;              // node index strides along y and z (nx, nx ny)
  float fx, fy, fz;
  bool free_x, free_y, free_z;
};

__device__ __forceinline__ float grid_axis(float x, float lo, float scale, int n, int& i, bool& free) {
  float u = (x - lo) * scale;
  const float top = (float)(n - 1);
  free = u >= 0.0f && u <= top;
  u = fminf(fmaxf(u, 0.0f), top);
  i = min((int)u, n - 2);
  return u - (float)i;
}

__device__ __forceinline__ GridCell grid_cell(const MediumView& g, float3 x) {
  GridCell c;
  int i, j, k;
  c.fx = grid_axis(x.x, g.lo.x, g.scale.x, g.nx, i, c.free_x);
  c.fy = grid_axis(x.y, g.lo.y, g.scale.y, g.ny, j, c.free_y);
  c.fz = grid_axis(x.z, g.lo.z, g.scale.z, g.nz, k, c.free_z);
  c.sx = g.nx;
  c.sy = g.nx * g.ny;
  c.base = ((size_t)k * g.ny + j) * g.nx + i;
  return c;
}

// The eight corner values of a cell (xyz of the float4 nodes).
struct CellNodes {
  float3 c000, c100, c010, c110, c001, c101, c011, c111;
};

__device__ __forceinline__ CellNodes cell_nodes(const MediumView& g, const GridCell& c) {
  const float4* p = g.mu + c.base;
  CellNodes q;
  q.c000 = xyz(__ldg(p));
  q.c100 = xyz(__ldg(p + 1));
  q.c010 = xyz(__ldg(p + c.sx));
  q.c110 = xyz(__ldg(p + c.sx + 1));
  q.c001 = xyz(__ldg(p + c.sy));
  q.c101 = xyz(__ldg(p + c.sy + 1));
  q.c011 = xyz(__ldg(p + c.sy + c.sx));
  q.c111 = xyz(__ldg(p + c.sy + c.sx + 1));
  return q;
}

__device__ __forceinline__ float3 lerp3(float3 a, float3 b, float f) { return a + (b - a) * f; }

// G at the cell position.
__device__ __forceinline__ float3 trilinear(const CellNodes& q, const GridCell& c) {
  const float3 x00 = lerp3(q.c000, q.c100, c.fx), x10 = lerp3(q.c010, q.c110, c.fx);
  const float3 x01 = lerp3(q.c001, q.c101, c.fx), x11 = lerp3(q.c011, q.c111, c.fx);
  return lerp3(lerp3(x00, x10, c.fy), lerp3(x01, x11, c.fy), c.fz);
}

// dG_c/dx_a for the three channels c: columns gx, gy, gz (each a float3 over
// the channels), zero along clamped axes.
__device__ __forceinline__ void trilinear_grad(const CellNodes& q, const GridCell& c, float3 scale, float3& gx,
                                               float3& gy, float3& gz) {
  const float ux = 1.0f - c.fx, uy = 1.0f - c.fy, uz = 1.0f - c.fz;
  gx = ((q.c100 - q.c000) * (uy * uz) + (q.c110 - q.c010) * (c.fy * uz) + (q.c101 - q.c001) * (uy * c.fz) +
        (q.c111 - q.c011) * (c.fy * c.fz)) * (c.free_x ? scale.x : 0.0f);
  gy = ((q.c010 - q.c000) * (ux * uz) + (q.c110 - q.c100) * (c.fx * uz) + (q.c011 - q.c001) * (ux * c.fz) +
        (q.c111 - q.c101) * (c.fx * c.fz)) * (c.free_y ? scale.y : 0.0f);
  gz = ((q.c001 - q.c000) * (ux * uy) + (q.c101 - q.c100) * (c.fx * uy) + (q.c011 - q.c010) * (ux * c.fy) +
        (q.c111 - q.c110) * (c.fx * c.fy)) * (c.free_z ? scale.z : 0.0f);
}

// Number of full steps of a segment of length t.
__device__ __forceinline__ int medium_full_steps(float t, float h) {
  const float m = floorf(t / h);
  if (!(m > 0.0f)) return 0;  // also a NaN length
  return m >= (float)kMaxMediumSteps ? kMaxMediumSteps : (int)m;
}

// Optical depth of the grid over o + s d, s in [0, t].
__device__ __forceinline__ float3 medium_depth(const MediumView& g, float3 o, float3 d, float t) {
  const float h = g.step;
  const int m = medium_full_steps(t, h);
  float3 sum = mk(0.f, 0.f, 0.f);
  for (int i = 0; i < m; ++i) {
    const GridCell c = grid_cell(g, o + d * (((float)i + 0.5f) * h));
    sum = sum + trilinear(cell_nodes(g, c), c) * h;
  }
  const float r = t - (float)m * h;
  const GridCell c = grid_cell(g, o + d * ((float)m * h + 0.5f * r));
  return sum + trilinear(cell_nodes(g, c), c) * r;
}

// dS/dt per channel (only the partial last step depends on t).
__device__ __forceinline__ float3 medium_depth_dt(const MediumView& g, float3 o, float3 d, float t) {
  const float h = g.step;
  const int m = medium_full_steps(t, h);
  const float r = t - (float)m * h;
  const GridCell c = grid_cell(g, o + d * ((float)m * h + 0.5f * r));
  const CellNodes q = cell_nodes(g, c);
  float3 gx, gy, gz;
  trilinear_grad(q, c, g.scale, gx, gy, gz);
  return trilinear(q, c) + (gx * d.x + gy * d.y + gz * d.z) * (0.5f * r);
}

// One 128-bit vector atomic per node (w unused).
__device__ __forceinline__ void medium_atomic4(float4* p, float3 v) {
  atomicAdd(p, make_float4(v.x, v.y, v.z, 0.f));
}

// Adjoint of the optical depth at fixed t: sbar = dJ/dS (per channel, one
// value for the whole segment).  Adds dJ/do and dJ/dd to obar and dbar and,
// when dmu is given, dJ/dG at the nodes: sbar times the sum over samples of
// w_i times the corner's trilinear weight.  Since sbar is constant along the
// segment, only those scalar sums are kept per corner, over consecutive
// samples in the same cell (a step of half a cell puts about two samples in
// each cell a ray crosses), and added with one atomic per node when the ray
// leaves the cell.  The sample gradient needs only sbar . G at the corners.
__device__ __forceinline__ void medium_flush(float4* p, int sx, int sy, float3 sbar, const float* acc) {
  medium_atomic4(p, sbar * acc[0]);
  medium_atomic4(p + 1, sbar * acc[1]);
  medium_atomic4(p + sx, sbar * acc[2]);
  medium_atomic4(p + sx + 1, sbar * acc[3]);
  medium_atomic4(p + sy, sbar * acc[4]);
  medium_atomic4(p + sy + 1, sbar * acc[5]);
  medium_atomic4(p + sy + sx, sbar * acc[6]);
  medium_atomic4(p + sy + sx + 1, sbar * acc[7]);
}

__device__ __forceinline__ void medium_backward(const MediumView& g, float4* dmu, float3 o, float3 d, float t,
                                                float3 sbar, float3& obar, float3& dbar) {
  const float h = g.step;
  const int m = medium_full_steps(t, h);
  const float r = t - (float)m * h;
  const int sx = g.nx, sy = g.nx * g.ny;
  float acc[8];
  size_t cur = ~(size_t)0;
  for (int i = 0; i <= m; ++i) {
    const float w = i < m ? h : r;
    const float s = i < m ? ((float)i + 0.5f) * h : (float)m * h + 0.5f * r;
    const GridCell c = grid_cell(g, o + d * s);
    const float4* p = g.mu + c.base;
    // sbar . G at the eight corners
    const float s000 = dot(sbar, xyz(__ldg(p))), s100 = dot(sbar, xyz(__ldg(p + 1)));
    const float s010 = dot(sbar, xyz(__ldg(p + sx))), s110 = dot(sbar, xyz(__ldg(p + sx + 1)));
    const float s001 = dot(sbar, xyz(__ldg(p + sy))), s101 = dot(sbar, xyz(__ldg(p + sy + 1)));
    const float s011 = dot(sbar, xyz(__ldg(p + sy + sx))), s111 = dot(sbar, xyz(__ldg(p + sy + sx + 1)));
    const float ux = 1.0f - c.fx, uy = 1.0f - c.fy, uz = 1.0f - c.fz;
    const float3 gp =
        mk(((s100 - s000) * (uy * uz) + (s110 - s010) * (c.fy * uz) + (s101 - s001) * (uy * c.fz) +
            (s111 - s011) * (c.fy * c.fz)) * (c.free_x ? g.scale.x : 0.0f),
           ((s010 - s000) * (ux * uz) + (s110 - s100) * (c.fx * uz) + (s011 - s001) * (ux * c.fz) +
            (s111 - s101) * (c.fx * c.fz)) * (c.free_y ? g.scale.y : 0.0f),
           ((s001 - s000) * (ux * uy) + (s101 - s100) * (c.fx * uy) + (s011 - s010) * (ux * c.fy) +
            (s111 - s110) * (c.fx * c.fy)) * (c.free_z ? g.scale.z : 0.0f)) * w;  // w dJ/dx at this sample
    obar = obar + gp;
    dbar = dbar + gp * s;
    if (dmu) {
      if (c.base != cur) {
        if (cur != ~(size_t)0) medium_flush(dmu + cur, sx, sy, sbar, acc);
        cur = c.base;
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q] = 0.f;
      }
      acc[0] += w * (ux * uy * uz);
      acc[1] += w * (c.fx * uy * uz);
      acc[2] += w * (ux * c.fy * uz);
      acc[3] += w * (c.fx * c.fy * uz);
      acc[4] += w * (ux * uy * c.fz);
      acc[5] += w * (c.fx * uy * c.fz);
      acc[6] += w * (ux * c.fy * c.fz);
      acc[7] += w * (c.fx * c.fy * c.fz);
    }
  }
  if (dmu && cur != ~(size_t)0) medium_flush(dmu + cur, sx, sy, sbar, acc);
}

}  // namespace dt

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
//
// G may instead be a multi-resolution hash texture (Sec. 3.3's 3D texture
// after Instant-NGP): the sum over up to 16 levels of the trilinear
// interpolation of a cubic lattice over the same box, whose corners are
// entries of the level's table slice, dense when the lattice fits it and
// otherwise at Instant-NGP's spatial hash.  Every sum above then runs level
// by level: the same steps, each level's cell and weights, its own scale.
#pragma once

#include "dt_internal.cuh"

namespace dt {

constexpr int kMaxMediumSteps = 8192;

struct MediumView {
  const float4* mu;
  int nx, ny, nz;
  float3 lo, scale;
  float step;
  int levels;             // hash texture levels (0: the dense grid)
  const GridLevel* lev;   // their descriptors, in the workspace's copy of the scene entry
};

// E: the scene entry as the kernel reads it (a kernel parameter or the
// table); Eg: the same entry in the workspace table, whose level array is
// indexed at run time.
__device__ __forceinline__ MediumView medium_view(const SceneEntry& E, const SceneEntry* Eg) {
  return MediumView{E.mu, E.gnx, E.gny, E.gnz, mk(E.glo_x, E.glo_y, E.glo_z),
                    mk(E.gscale_x, E.gscale_y, E.gscale_z), E.gstep, E.glevels, Eg->glev};
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
template <class Cell>
__device__ __forceinline__ float3 trilinear(const CellNodes& q, const Cell& c) {
  const float3 x00 = lerp3(q.c000, q.c100, c.fx), x10 = lerp3(q.c010, q.c110, c.fx);
  const float3 x01 = lerp3(q.c001, q.c101, c.fx), x11 = lerp3(q.c011, q.c111, c.fx);
  return lerp3(lerp3(x00, x10, c.fy), lerp3(x01, x11, c.fy), c.fz);
}

// dG_c/dx_a for the three channels c: columns gx, gy, gz (each a float3 over
// the channels), zero along clamped axes.
template <class Cell>
__device__ __forceinline__ void trilinear_grad(const CellNodes& q, const Cell& c, float3 scale, float3& gx,
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

// ---------------------------------------------------------------------------
// hash texture
// ---------------------------------------------------------------------------
// Instant-NGP's spatial hash of a lattice point (Mueller et al. 2022, Eq. 4
// with d = 3): XOR of the coordinates times 1, 2654435761 and 805459861 in
// 32-bit arithmetic; the level keeps its low bits (tables are powers of two).
__device__ __forceinline__ uint32_t ingp_hash(uint32_t i, uint32_t j, uint32_t k) {
  return i ^ (j * 2654435761u) ^ (k * 805459861u);
}

// A level's cell containing x: fractions and clamping as grid_cell, and the
// lattice coordinates of its (0, 0, 0) corner.
struct LevelCell {
  uint32_t i, j, k;
  float fx, fy, fz;
  bool free_x, free_y, free_z;
};

__device__ __forceinline__ LevelCell level_cell(const GridLevel& L, float3 lo, float3 x) {
  LevelCell c;
  int i, j, k;
  c.fx = grid_axis(x.x, lo.x, L.sx, L.n, i, c.free_x);
  c.fy = grid_axis(x.y, lo.y, L.sy, L.n, j, c.free_y);
  c.fz = grid_axis(x.z, lo.z, L.sz, L.n, k, c.free_z);
  c.i = (uint32_t)i;
  c.j = (uint32_t)j;
  c.k = (uint32_t)k;
  return c;
}

// Table entry of the level's lattice point (i, j, k).
__device__ __forceinline__ uint32_t level_entry(const GridLevel& L, uint32_t i, uint32_t j, uint32_t k) {
  const uint32_t n = (uint32_t)L.n;
  return L.off + (L.mask ? (ingp_hash(i, j, k) & L.mask) : ((k * n + j) * n + i));
}

// Corner q (x fastest, then y, then z) of the cell at (i, j, k).
__device__ __forceinline__ uint32_t corner_entry(const GridLevel& L, uint32_t i, uint32_t j, uint32_t k, int q) {
  return level_entry(L, i + (uint32_t)(q & 1), j + (uint32_t)((q >> 1) & 1), k + (uint32_t)(q >> 2));
}

__device__ __forceinline__ CellNodes level_nodes(const float4* mu, const GridLevel& L, const LevelCell& c) {
  CellNodes q;
  q.c000 = xyz(__ldg(mu + corner_entry(L, c.i, c.j, c.k, 0)));
  q.c100 = xyz(__ldg(mu + corner_entry(L, c.i, c.j, c.k, 1)));
  q.c010 = xyz(__ldg(mu + corner_entry(L, c.i, c.j, c.k, 2)));
  q.c110 = xyz(__ldg(mu + corner_entry(L, c.i, c.j, c.k, 3)));
  q.c001 = xyz(__ldg(mu + corner_entry(L, c.i, c.j, c.k, 4)));
  q.c101 = xyz(__ldg(mu + corner_entry(L, c.i, c.j, c.k, 5)));
  q.c011 = xyz(__ldg(mu + corner_entry(L, c.i, c.j, c.k, 6)));
  q.c111 = xyz(__ldg(mu + corner_entry(L, c.i, c.j, c.k, 7)));
  return q;
}

__device__ __forceinline__ GridLevel load_level(const GridLevel* p) {
  GridLevel L;
  const int4 a = __ldg(reinterpret_cast<const int4*>(p));
  const int4 b = __ldg(reinterpret_cast<const int4*>(p) + 1);
  L.n = a.x;
  L.mask = (uint32_t)a.y;
  L.off = (uint32_t)a.z;
  L.sx = __int_as_float(a.w);
  L.sy = __int_as_float(b.x);
  L.sz = __int_as_float(b.y);
  L.pad[0] = L.pad[1] = 0;
  return L;
}

// Optical depth of the hash texture over o + s d, s in [0, t]: the steps of
// medium_depth, level by level.
__device__ __forceinline__ float3 hash_depth(const MediumView& g, float3 o, float3 d, float t) {
  const float h = g.step;
  const int m = medium_full_steps(t, h);
  const float r = t - (float)m * h;
  float3 sum = mk(0.f, 0.f, 0.f);
  for (int l = 0; l < g.levels; ++l) {
    const GridLevel L = load_level(g.lev + l);
    for (int i = 0; i <= m; ++i) {
      const float w = i < m ? h : r;
      const float s = i < m ? ((float)i + 0.5f) * h : (float)m * h + 0.5f * r;
      const LevelCell c = level_cell(L, g.lo, o + d * s);
      sum = sum + trilinear(level_nodes(g.mu, L, c), c) * w;
    }
  }
  return sum;
}

__device__ __forceinline__ float3 hash_depth_dt(const MediumView& g, float3 o, float3 d, float t) {
  const float h = g.step;
  const int m = medium_full_steps(t, h);
  const float r = t - (float)m * h;
  const float3 x = o + d * ((float)m * h + 0.5f * r);
  float3 sum = mk(0.f, 0.f, 0.f);
  for (int l = 0; l < g.levels; ++l) {
    const GridLevel L = load_level(g.lev + l);
    const LevelCell c = level_cell(L, g.lo, x);
    const CellNodes q = level_nodes(g.mu, L, c);
    float3 gx, gy, gz;
    trilinear_grad(q, c, mk(L.sx, L.sy, L.sz), gx, gy, gz);
    sum = sum + trilinear(q, c) + (gx * d.x + gy * d.y + gz * d.z) * (0.5f * r);
  }
  return sum;
}

// Optical depth of the grid over o + s d, s in [0, t] (kHash: the scene may
// hold a hash texture instead; without it that code is not compiled).
template <bool kHash>
__device__ __forceinline__ float3 medium_depth(const MediumView& g, float3 o, float3 d, float t) {
  if (kHash && g.levels) return hash_depth(g, o, d, t);
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
template <bool kHash>
__device__ __forceinline__ float3 medium_depth_dt(const MediumView& g, float3 o, float3 d, float t) {
  if (kHash && g.levels) return hash_depth_dt(g, o, d, t);
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

// The adjoint of hash_depth, level by level as medium_backward below: per
// sample the gradient of sbar . G_l from sbar . (corner values), per cell
// the scalar weight sums, flushed into the cell's eight entries (hashed
// corners that share an entry add) when the ray leaves the cell.
__device__ __forceinline__ void hash_flush(float4* dmu, const GridLevel& L, uint32_t i, uint32_t j, uint32_t k,
                                           float3 sbar, const float* acc) {
#pragma unroll
  for (int q = 0; q < 8; ++q) medium_atomic4(dmu + corner_entry(L, i, j, k, q), sbar * acc[q]);
}

__device__ __forceinline__ void hash_backward(const MediumView& g, float4* dmu, float3 o, float3 d, float t,
                                              float3 sbar, float3& obar, float3& dbar) {
  const float h = g.step;
  const int m = medium_full_steps(t, h);
  const float r = t - (float)m * h;
  for (int l = 0; l < g.levels; ++l) {
    const GridLevel L = load_level(g.lev + l);
    float acc[8];
    uint32_t pi = ~0u, pj = 0, pk = 0;  // the cell whose sums are pending (pi = ~0: none)
    for (int i = 0; i <= m; ++i) {
      const float w = i < m ? h : r;
      const float s = i < m ? ((float)i + 0.5f) * h : (float)m * h + 0.5f * r;
      const LevelCell c = level_cell(L, g.lo, o + d * s);
      float sv[8];  // sbar . G at the eight corners
#pragma unroll
      for (int q = 0; q < 8; ++q) sv[q] = dot(sbar, xyz(__ldg(g.mu + corner_entry(L, c.i, c.j, c.k, q))));
      const float ux = 1.0f - c.fx, uy = 1.0f - c.fy, uz = 1.0f - c.fz;
      const float3 gp =
          mk(((sv[1] - sv[0]) * (uy * uz) + (sv[3] - sv[2]) * (c.fy * uz) + (sv[5] - sv[4]) * (uy * c.fz) +
              (sv[7] - sv[6]) * (c.fy * c.fz)) * (c.free_x ? L.sx : 0.0f),
             ((sv[2] - sv[0]) * (ux * uz) + (sv[3] - sv[1]) * (c.fx * uz) + (sv[6] - sv[4]) * (ux * c.fz) +
              (sv[7] - sv[5]) * (c.fx * c.fz)) * (c.free_y ? L.sy : 0.0f),
             ((sv[4] - sv[0]) * (ux * uy) + (sv[5] - sv[1]) * (c.fx * uy) + (sv[6] - sv[2]) * (ux * c.fy) +
              (sv[7] - sv[3]) * (c.fx * c.fy)) * (c.free_z ? L.sz : 0.0f)) * w;
      obar = obar + gp;
      dbar = dbar + gp * s;
      if (dmu) {
        if (c.i != pi || c.j != pj || c.k != pk) {
          if (pi != ~0u) hash_flush(dmu, L, pi, pj, pk, sbar, acc);
          pi = c.i;
          pj = c.j;
          pk = c.k;
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
    if (dmu && pi != ~0u) hash_flush(dmu, L, pi, pj, pk, sbar, acc);
  }
}

template <bool kHash>
__device__ __forceinline__ void medium_backward(const MediumView& g, float4* dmu, float3 o, float3 d, float t,
                                                float3 sbar, float3& obar, float3& dbar) {
  if (kHash && g.levels) {
    hash_backward(g, dmu, o, d, t, sbar, obar, dbar);
    return;
  }
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

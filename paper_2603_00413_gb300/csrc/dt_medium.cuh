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
  c.base = ((uint32_t)k * (uint32_t)g.ny + (uint32_t)j) * (uint32_t)g.nx + (uint32_t)i;  // < 2^31 nodes (checked)
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
constexpr uint32_t kHashPrimeY = 2654435761u, kHashPrimeZ = 805459861u;

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

// The table entries of the eight corners of a level's cell at lattice point
// (i, j, k), corner q = (i + (q & 1), j + ((q >> 1) & 1), k + (q >> 2)):
// the level's first entry plus, when the lattice fits the table, the dense
// index (k n + j) n + i (so the corners add 0, 1, n, n + 1, n^2, ...), else
// the spatial hash masked to the table, with the per-axis terms formed once
// ((j + 1) kHashPrimeY = j kHashPrimeY + kHashPrimeY in 32-bit arithmetic,
// likewise for k), so each corner is one three-way XOR, a mask and an add.
__device__ __forceinline__ void level_corner_entries(const GridLevel& L, const LevelCell& c, size_t (&e)[8]) {
  if (L.mask) {
    const uint32_t x0 = c.i, x1 = c.i + 1u;
    const uint32_t y0 = c.j * kHashPrimeY, y1 = y0 + kHashPrimeY;
    const uint32_t z0 = c.k * kHashPrimeZ, z1 = z0 + kHashPrimeZ;
    e[0] = L.off + ((x0 ^ y0 ^ z0) & L.mask);
    e[1] = L.off + ((x1 ^ y0 ^ z0) & L.mask);
    e[2] = L.off + ((x0 ^ y1 ^ z0) & L.mask);
    e[3] = L.off + ((x1 ^ y1 ^ z0) & L.mask);
    e[4] = L.off + ((x0 ^ y0 ^ z1) & L.mask);
    e[5] = L.off + ((x1 ^ y0 ^ z1) & L.mask);
    e[6] = L.off + ((x0 ^ y1 ^ z1) & L.mask);
    e[7] = L.off + ((x1 ^ y1 ^ z1) & L.mask);
  } else {
    const uint32_t n = (uint32_t)L.n, b = L.off + (c.k * n + c.j) * n + c.i, nn = n * n;
    e[0] = b; e[1] = b + 1u; e[2] = b + n; e[3] = b + n + 1u;
    e[4] = b + nn; e[5] = b + nn + 1u; e[6] = b + nn + n; e[7] = b + nn + n + 1u;
  }
}

__device__ __forceinline__ CellNodes level_nodes(const float4* mu, const GridLevel& L, const LevelCell& c) {
  size_t e[8];
  level_corner_entries(L, c, e);
  CellNodes q;
  q.c000 = xyz(__ldg(mu + e[0]));
  q.c100 = xyz(__ldg(mu + e[1]));
  q.c010 = xyz(__ldg(mu + e[2]));
  q.c110 = xyz(__ldg(mu + e[3]));
  q.c001 = xyz(__ldg(mu + e[4]));
  q.c101 = xyz(__ldg(mu + e[5]));
  q.c011 = xyz(__ldg(mu + e[6]));
  q.c111 = xyz(__ldg(mu + e[7]));
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

template <bool kHash>
__device__ __forceinline__ void medium_scatter(const MediumView& g, float4* dmu, float3 o, float3 d, float t,
                                               float3 sbar);

// The samples' share of the adjoint of hash_depth, level by level: per
// sample the gradient of sbar . G_l from sbar . (corner values).
__device__ __forceinline__ void hash_backward(const MediumView& g, float3 o, float3 d, float t, float3 sbar,
                                              float3& obar, float3& dbar) {
  const float h = g.step;
  const int m = medium_full_steps(t, h);
  const float r = t - (float)m * h;
  for (int l = 0; l < g.levels; ++l) {
    const GridLevel L = load_level(g.lev + l);
    for (int i = 0; i <= m; ++i) {
      const float w = i < m ? h : r;
      const float s = i < m ? ((float)i + 0.5f) * h : (float)m * h + 0.5f * r;
      const LevelCell c = level_cell(L, g.lo, o + d * s);
      float sv[8];  // sbar . G at the eight corners
      size_t e[8];
      level_corner_entries(L, c, e);
#pragma unroll
      for (int q = 0; q < 8; ++q) sv[q] = dot(sbar, xyz(__ldg(g.mu + e[q])));
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
    }
  }
}

// Adjoint of the optical depth at fixed t: sbar = dJ/dS (per channel, one
// value for the whole segment).  Adds dJ/do and dJ/dd to obar and dbar
// (the samples move with o and d; the gradient of sbar . G needs only sbar .
// G at each sample's corners) and, when dmu is given, dJ/dG at the nodes or
// entries (medium_scatter).
template <bool kHash>
__device__ __forceinline__ void medium_backward(const MediumView& g, float4* dmu, float3 o, float3 d, float t,
                                                float3 sbar, float3& obar, float3& dbar) {
  if (kHash && g.levels) {
    hash_backward(g, o, d, t, sbar, obar, dbar);
  } else {
    const float h = g.step;
    const int m = medium_full_steps(t, h);
    const float r = t - (float)m * h;
    const int sx = g.nx, sy = g.nx * g.ny;
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
    }
  }
  if (dmu) medium_scatter<kHash>(g, dmu, o, d, t, sbar);
}

// ---------------------------------------------------------------------------
// tape_mode 2: the medium's moments in the forward, its scatter in the backward
// ---------------------------------------------------------------------------
// Everything the backward needs of the optical depth S over o + s d, s in
// [0, t], at fixed t: S; dS/dt (the partial last step, as medium_depth_dt);
// and the motion of the samples with o and d, whose adjoint is linear in
// sbar = dJ/dS:
//   dJ/do = sum_c sbar_c Do[c],  Do[c] = sum_i w_i grad G_c(x_i),
//   dJ/dd = sum_c sbar_c Dd[c],  Dd[c] = sum_i w_i s_i grad G_c(x_i),
// so the forward, which reads the corner values of every sample anyway,
// keeps the two 3x3 sums and the backward needs no corner value at all.
// gx, gy, gz of trilinear_grad are the columns dG/dx_a over the channels.
//
// The scatter of dJ/dG into the medium walks each level's cells along the
// segment.  Consecutive samples share their cell, or step to a neighbouring
// cell (at most one cell along each axis) with which it shares a face, an
// edge or a vertex: the corners the two cells share keep their pending
// weight sums, and only the corners the step leaves behind are flushed with
// an atomic -- on the bench's hash texture about 40 % fewer atomics than
// flushing the whole cell at every change.
struct MediumMoments {
  float3 S, dt;
  float3 ox, oy, oz;  // columns of Do: dS/do_x, dS/do_y, dS/do_z (each over the channels)
  float3 dx, dy, dz;  // columns of Dd
};

__device__ __forceinline__ void moments_sample(MediumMoments& M, float3 G, float3 gx, float3 gy, float3 gz, float w,
                                               float s) {
  M.S = M.S + G * w;
  M.ox = M.ox + gx * w;
  M.oy = M.oy + gy * w;
  M.oz = M.oz + gz * w;
  const float ws = w * s;
  M.dx = M.dx + gx * ws;
  M.dy = M.dy + gy * ws;
  M.dz = M.dz + gz * ws;
}

// Corner q of a cell is (q & 1, (q >> 1) & 1, q >> 2).  For a step by
// (dx, dy, dz), each in {-1, 0, 1}: the old corners the new cell does not
// hold, and the new corners the old cell did not hold.
__device__ __forceinline__ unsigned corners_left(int dx, int dy, int dz) {
  return (dx > 0 ? 0x55u : 0u) | (dx < 0 ? 0xAAu : 0u) | (dy > 0 ? 0x33u : 0u) | (dy < 0 ? 0xCCu : 0u) |
         (dz > 0 ? 0x0Fu : 0u) | (dz < 0 ? 0xF0u : 0u);
}
__device__ __forceinline__ unsigned corners_added(int dx, int dy, int dz) {
  return (dx > 0 ? 0xAAu : 0u) | (dx < 0 ? 0x55u : 0u) | (dy > 0 ? 0xCCu : 0u) | (dy < 0 ? 0x33u : 0u) |
         (dz > 0 ? 0xF0u : 0u) | (dz < 0 ? 0x0Fu : 0u);
}

// Moves the per-corner values of the old cell to the corners they are in
// the new one (the added corners keep stale values: the caller refills or
// clears them).  Axis by axis over the pairs of corners that differ in it.
template <class T>
__device__ __forceinline__ void shift_pairs(T (&v)[8], int dl, int bit) {
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    if (q & bit) continue;
    const T a = v[q], b = v[q | bit];
    v[q] = dl > 0 ? b : a;
    v[q | bit] = dl < 0 ? a : b;
  }
}
template <class T>
__device__ __forceinline__ void shift_corners(T (&v)[8], int dx, int dy, int dz) {
  shift_pairs(v, dx, 1);
  shift_pairs(v, dy, 2);
  shift_pairs(v, dz, 4);
}

__device__ __forceinline__ bool one_step(int dx, int dy, int dz) {
  return dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1 && dz >= -1 && dz <= 1;
}

// Lattice coordinates of the dense grid's cell (clamping as grid_cell).
struct GridIJK {
  int i, j, k;
  float fx, fy, fz;
  bool free_x, free_y, free_z;
};
__device__ __forceinline__ GridIJK grid_ijk(const MediumView& g, float3 x) {
  GridIJK c;
  c.fx = grid_axis(x.x, g.lo.x, g.scale.x, g.nx, c.i, c.free_x);
  c.fy = grid_axis(x.y, g.lo.y, g.scale.y, g.ny, c.j, c.free_y);
  c.fz = grid_axis(x.z, g.lo.z, g.scale.z, g.nz, c.k, c.free_z);
  return c;
}
__device__ __forceinline__ uint32_t grid_corner(const MediumView& g, int i, int j, int k, int q) {
  return ((uint32_t)(k + (q >> 2)) * (uint32_t)g.ny + (uint32_t)(j + ((q >> 1) & 1))) * (uint32_t)g.nx +
         (uint32_t)(i + (q & 1));
}

// G and its gradient together, sharing the interpolation's intermediate
// values: the differences along x feed both the x interpolations and
// dG/dx, the differences of the x-interpolated values along y feed the y
// interpolations and dG/dy, and the difference of the two y-interpolated
// values along z gives G and dG/dz (the derivatives of trilinear; about
// half of the arithmetic of trilinear and trilinear_grad apart).
template <class Cell>
__device__ __forceinline__ float3 trilinear_value_grad(const CellNodes& q, const Cell& c, float3 scale, float3& gx,
                                                       float3& gy, float3& gz) {
  const float3 a00 = q.c100 - q.c000, a10 = q.c110 - q.c010, a01 = q.c101 - q.c001, a11 = q.c111 - q.c011;
  const float3 x00 = q.c000 + a00 * c.fx, x10 = q.c010 + a10 * c.fx;
  const float3 x01 = q.c001 + a01 * c.fx, x11 = q.c011 + a11 * c.fx;
  const float3 b0 = x10 - x00, b1 = x11 - x01;
  const float3 y0 = x00 + b0 * c.fy, y1 = x01 + b1 * c.fy;
  const float3 e = y1 - y0;
  const float3 ax0 = a00 + (a10 - a00) * c.fy, ax1 = a01 + (a11 - a01) * c.fy;
  gx = (ax0 + (ax1 - ax0) * c.fz) * (c.free_x ? scale.x : 0.0f);
  gy = (b0 + (b1 - b0) * c.fz) * (c.free_y ? scale.y : 0.0f);
  gz = e * (c.free_z ? scale.z : 0.0f);
  return y0 + e * c.fz;
}

// One level's (or the dense grid's) samples for the forward: each sample's
// eight corner values, its G and gradient into the moments.  (Carrying the
// shared corners' values from cell to cell, as the scatter below carries its
// sums, read 60 % fewer entries but made this pass twice as slow: the
// per-sample reads are independent of one another, the carried ones are
// not.)
template <class Cell, class Entry>
__device__ __forceinline__ void moments_walk(MediumMoments& M, const float4* mu, float3 o, float3 d, float h, int m,
                                             float r, float3 scale, const Cell& cell_of, const Entry& entry_of) {
  for (int i = 0; i <= m; ++i) {
    const float w = i < m ? h : r;
    const float s = i < m ? ((float)i + 0.5f) * h : (float)m * h + 0.5f * r;
    const auto c = cell_of(o + d * s);
    size_t e[8];
    entry_of(c, e);
    CellNodes qn;
    qn.c000 = xyz(__ldg(mu + e[0]));
    qn.c100 = xyz(__ldg(mu + e[1]));
    qn.c010 = xyz(__ldg(mu + e[2]));
    qn.c110 = xyz(__ldg(mu + e[3]));
    qn.c001 = xyz(__ldg(mu + e[4]));
    qn.c101 = xyz(__ldg(mu + e[5]));
    qn.c011 = xyz(__ldg(mu + e[6]));
    qn.c111 = xyz(__ldg(mu + e[7]));
    float3 gx, gy, gz;
    const float3 G = trilinear_value_grad(qn, c, scale, gx, gy, gz);
    moments_sample(M, G, gx, gy, gz, w, s);
    if (i == m) M.dt = M.dt + G + (gx * d.x + gy * d.y + gz * d.z) * (0.5f * r);
  }
}

template <bool kHash>
__device__ __forceinline__ MediumMoments medium_moments(const MediumView& g, float3 o, float3 d, float t) {
  const float h = g.step;
  const int m = medium_full_steps(t, h);
  const float r = t - (float)m * h;
  MediumMoments M;
  M.S = M.dt = M.ox = M.oy = M.oz = M.dx = M.dy = M.dz = mk(0.f, 0.f, 0.f);
  if (kHash && g.levels) {
    for (int l = 0; l < g.levels; ++l) {
      const GridLevel L = load_level(g.lev + l);
      moments_walk(M, g.mu, o, d, h, m, r, mk(L.sx, L.sy, L.sz),
                   [&](float3 x) { return level_cell(L, g.lo, x); },
                   [&](const LevelCell& c, size_t (&e)[8]) { level_corner_entries(L, c, e); });
    }
    return M;
  }
  moments_walk(M, g.mu, o, d, h, m, r, g.scale, [&](float3 x) { return grid_ijk(g, x); },
               [&](const GridIJK& c, size_t (&e)[8]) {
                 const uint32_t b = grid_corner(g, c.i, c.j, c.k, 0), sx = (uint32_t)g.nx, sy = sx * (uint32_t)g.ny;
                 e[0] = b; e[1] = b + 1; e[2] = b + sx; e[3] = b + sx + 1;
                 e[4] = b + sy; e[5] = b + sy + 1; e[6] = b + sy + sx; e[7] = b + sy + sx + 1;
               });
  return M;
}

// dJ/dG at the table entries (or grid nodes) for one segment: sbar times
// the sum over samples of w_i times each corner's trilinear weight.  The
// sums are kept per corner of the current cell and carried along shared
// corners; a corner is added to its entry with one 128-bit atomic when the
// walk leaves it (hashed corners that share an entry add).
template <class Cell, class Entry>
__device__ __forceinline__ void scatter_walk(float4* dmu, float3 o, float3 d, float h, int m, float r, float3 sbar,
                                             const Cell& cell_of, const Entry& entry_of) {
  float acc[8];
  int pi = 0, pj = 0, pk = 0;
  bool have = false;
  for (int i = 0; i <= m; ++i) {
    const float w = i < m ? h : r;
    const float s = i < m ? ((float)i + 0.5f) * h : (float)m * h + 0.5f * r;
    const auto c = cell_of(o + d * s);
    const int dx = (int)c.i - pi, dy = (int)c.j - pj, dz = (int)c.k - pk;
    if (!have || dx || dy || dz) {
      unsigned fresh = 0xFFu;
      if (have) {
        const bool near = one_step(dx, dy, dz);
        const unsigned left = near ? corners_left(dx, dy, dz) : 0xFFu;
        size_t e[8];
        entry_of(pi, pj, pk, e);
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (left & (1u << q)) medium_atomic4(dmu + e[q], sbar * acc[q]);
        if (near) {
          shift_corners(acc, dx, dy, dz);
          fresh = corners_added(dx, dy, dz);
        }
      }
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (fresh & (1u << q)) acc[q] = 0.f;
      have = true;
      pi = (int)c.i;
      pj = (int)c.j;
      pk = (int)c.k;
    }
    const float ux = 1.0f - c.fx, uy = 1.0f - c.fy, uz = 1.0f - c.fz;
    acc[0] += w * (ux * uy * uz);
    acc[1] += w * (c.fx * uy * uz);
    acc[2] += w * (ux * c.fy * uz);
    acc[3] += w * (c.fx * c.fy * uz);
    acc[4] += w * (ux * uy * c.fz);
    acc[5] += w * (c.fx * uy * c.fz);
    acc[6] += w * (ux * c.fy * c.fz);
    acc[7] += w * (c.fx * c.fy * c.fz);
  }
  if (have) {
    size_t e[8];
    entry_of(pi, pj, pk, e);
#pragma unroll
    for (int q = 0; q < 8; ++q) medium_atomic4(dmu + e[q], sbar * acc[q]);
  }
}

template <bool kHash>
__device__ __forceinline__ void medium_scatter(const MediumView& g, float4* dmu, float3 o, float3 d, float t,
                                               float3 sbar) {
  const float h = g.step;
  const int m = medium_full_steps(t, h);
  const float r = t - (float)m * h;
  if (kHash && g.levels) {
    for (int l = 0; l < g.levels; ++l) {
      const GridLevel L = load_level(g.lev + l);
      scatter_walk(dmu, o, d, h, m, r, sbar, [&](float3 x) { return level_cell(L, g.lo, x); },
                   [&](int i, int j, int k, size_t (&e)[8]) {
                     LevelCell c;
                     c.i = (uint32_t)i;
                     c.j = (uint32_t)j;
                     c.k = (uint32_t)k;
                     level_corner_entries(L, c, e);
                   });
    }
    return;
  }
  scatter_walk(dmu, o, d, h, m, r, sbar, [&](float3 x) { return grid_ijk(g, x); },
               [&](int i, int j, int k, size_t (&e)[8]) {
                 const uint32_t b = grid_corner(g, i, j, k, 0), sx = (uint32_t)g.nx, sy = sx * (uint32_t)g.ny;
                 e[0] = b; e[1] = b + 1; e[2] = b + sx; e[3] = b + sx + 1;
                 e[4] = b + sy; e[5] = b + sy + 1; e[6] = b + sy + sx; e[7] = b + sy + sx + 1;
               });
}

}  // namespace dt

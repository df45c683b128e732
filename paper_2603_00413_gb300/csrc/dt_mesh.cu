// The step after the gradient (DiffTrans App. A): the mesh's edge graph, the
// large-steps update with AdamUniform, and the edge-normal regulariser.
//
//  * Topology: the distinct neighbours of every vertex in CSR form, built on
//    the device from the triangles (count, scan, fill, sort and deduplicate
//    each vertex's list, scan, compact).
//  * Laplacian L = D - A of that graph (uniform weights); M = I + lambda L is
//    symmetric positive definite, applied matrix-free from the CSR.
//  * Solve M x = b (three right-hand sides) by conjugate gradients with the
//    diagonal 1 + lambda deg as preconditioner, at most a given number of
//    iterations (a column stops once its residual has fallen by 1e-6),
//    every scalar on the device (no host synchronisation).
//  * Large-steps update: u = M V; g_u = M^-1 dJ/dV; AdamUniform on u (one
//    second moment, the max of g_u^2); V = M^-1 u.
//  * L_edge = (1/|E|) sum over edges of (1 - n_i . n_j)^2 with n the unit
//    vertex normals; its gradient with respect to the Eq. 13 normals (the
//    caller chains it to the vertices with the normals' backward).
#include <cuda_runtime.h>
#include <stdint.h>

#include "dt_internal.cuh"

namespace dt {

// ---------------------------------------------------------------------------
// topology buffer
// ---------------------------------------------------------------------------
struct TopoHeader {
  int32_t nv, nf;
  int32_t nnz;      // directed neighbour entries (2 |E|), written on the device
  int32_t max_deg;  // largest neighbour count, written on the device
};

struct TopoLayout {
  size_t off_row, off_col, off_raw_cnt, off_raw_off, off_cursor, off_raw, total;
  TopoLayout(int32_t nv, int32_t nf) {
    size_t o = 256;
    auto take = [&](size_t bytes) { size_t r = o; o = align_up(o + bytes, 256); return r; };
    off_row = take(((size_t)nv + 1) * sizeof(int32_t));
    off_col = take((size_t)6 * nf * sizeof(int32_t));
    off_raw_cnt = take(((size_t)nv + 1) * sizeof(uint32_t));
    off_raw_off = take(((size_t)nv + 1) * sizeof(uint32_t));
    off_cursor = take((size_t)nv * sizeof(uint32_t));
    off_raw = take((size_t)6 * nf * sizeof(int32_t));
    total = o;
  }
};

struct TopoView {
  TopoHeader* hdr;
  int32_t* row;  // [nv + 1]
  int32_t* col;  // [nnz]
  uint32_t* raw_cnt;
  uint32_t* raw_off;
  uint32_t* cursor;
  int32_t* raw;
};

static TopoView topo_view(void* base, int32_t nv, int32_t nf) {
  TopoLayout L(nv, nf);
  char* b = (char*)base;
  return TopoView{(TopoHeader*)b, (int32_t*)(b + L.off_row), (int32_t*)(b + L.off_col),
                  (uint32_t*)(b + L.off_raw_cnt), (uint32_t*)(b + L.off_raw_off), (uint32_t*)(b + L.off_cursor),
                  (int32_t*)(b + L.off_raw)};
}

size_t topology_bytes(int32_t nv, int32_t nf) { return TopoLayout(nv, nf).total; }

static int blocks_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  const int64_t cap = 8 * (int64_t)num_sms();
  if (b > cap) b = cap;
  return (int)(b > 0 ? b : 1);
}

// every triangle lists each of its vertices' two other vertices
__global__ void k_topo_count(const int32_t* __restrict__ F, int32_t nf, int32_t nv, uint32_t* __restrict__ raw_cnt) {
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += gridDim.x * blockDim.x)
    for (int k = 0; k < 3; ++k) {
      const int v = F[3 * f + k];
      if (v >= 0 && v < nv) atomicAdd(raw_cnt + v, 2u);
    }
}

__global__ void k_topo_fill(const int32_t* __restrict__ F, int32_t nf, int32_t nv, const uint32_t* __restrict__ raw_off,
                            uint32_t* __restrict__ cursor, int32_t* __restrict__ raw) {
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += gridDim.x * blockDim.x) {
    const int a = F[3 * f], b = F[3 * f + 1], c = F[3 * f + 2];
    const int tri[3] = {a, b, c};
    for (int k = 0; k < 3; ++k) {
      const int v = tri[k];
      if (v < 0 || v >= nv) continue;
      const uint32_t at = raw_off[v] + atomicAdd(cursor + v, 2u);
      raw[at] = tri[(k + 1) % 3];
      raw[at + 1] = tri[(k + 2) % 3];
    }
  }
}

// sort each vertex's list (insertion sort: lists are a vertex's valence
// times two) and keep the distinct in-range entries other than the vertex
// itself at its front; raw_cnt[v] becomes the distinct count
__global__ void k_topo_dedupe(int32_t nv, const uint32_t* __restrict__ raw_off, uint32_t* __restrict__ raw_cnt,
                              int32_t* __restrict__ raw, TopoHeader* hdr) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x) {
    int32_t* l = raw + raw_off[v];
    const int n = (int)raw_cnt[v];
    for (int i = 1; i < n; ++i) {
      const int32_t x = l[i];
      int j = i - 1;
      while (j >= 0 && l[j] > x) {
        l[j + 1] = l[j];
        --j;
      }
      l[j + 1] = x;
    }
    int u = 0;
    for (int i = 0; i < n; ++i) {
      const int32_t x = l[i];
      if (x < 0 || x >= nv || x == v) continue;
      if (u > 0 && l[u - 1] == x) continue;
      l[u++] = x;
    }
    raw_cnt[v] = (uint32_t)u;
    atomicMax(&hdr->max_deg, u);
  }
}

__global__ void k_topo_compact(int32_t nv, const uint32_t* __restrict__ raw_off, const uint32_t* __restrict__ cnt,
                               const uint32_t* __restrict__ row_u, const int32_t* __restrict__ raw,
                               int32_t* __restrict__ row, int32_t* __restrict__ col, TopoHeader* hdr) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x) {
    const uint32_t o = row_u[v], n = cnt[v];
    row[v] = (int32_t)o;
    for (uint32_t i = 0; i < n; ++i) col[o + i] = raw[raw_off[v] + i];
    if (v == nv - 1) {
      row[nv] = (int32_t)(o + n);
      hdr->nnz = (int32_t)(o + n);
    }
  }
}

__global__ void k_topo_header(TopoHeader* hdr, int32_t nv, int32_t nf) {
  hdr->nv = nv;
  hdr->nf = nf;
  hdr->nnz = 0;
  hdr->max_deg = 0;
}

void launch_build_topology(const int32_t* F, int32_t nf, int32_t nv, void* topo, cudaStream_t s) {
  TopoView T = topo_view(topo, nv, nf);
  ProfScope ps("topology_build", s);
  k_topo_header<<<1, 1, 0, s>>>(T.hdr, nv, nf);
  cudaMemsetAsync(T.raw_cnt, 0, ((size_t)nv + 1) * sizeof(uint32_t), s);
  cudaMemsetAsync(T.cursor, 0, (size_t)nv * sizeof(uint32_t), s);
  k_topo_count<<<blocks_for(nf, 256), 256, 0, s>>>(F, nf, nv, T.raw_cnt);
  cudaMemcpyAsync(T.raw_off, T.raw_cnt, ((size_t)nv + 1) * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
  launch_scan_exclusive(T.raw_off, nv + 1, s);
  k_topo_fill<<<blocks_for(nf, 256), 256, 0, s>>>(F, nf, nv, T.raw_off, T.cursor, T.raw);
  k_topo_dedupe<<<blocks_for(nv, 128), 128, 0, s>>>(nv, T.raw_off, T.raw_cnt, T.raw, T.hdr);
  // distinct counts -> row starts (the cursor array, free now, holds the scan)
  cudaMemcpyAsync(T.cursor, T.raw_cnt, (size_t)nv * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
  launch_scan_exclusive(T.cursor, nv, s);
  k_topo_compact<<<blocks_for(nv, 256), 256, 0, s>>>(nv, T.raw_off, T.raw_cnt, T.cursor, T.raw, T.row, T.col,
                                                      T.hdr);
}

// ---------------------------------------------------------------------------
// M = I + lambda L, applied from the CSR; conjugate gradients
// ---------------------------------------------------------------------------
__device__ __forceinline__ float3 apply_m(const int32_t* __restrict__ row, const int32_t* __restrict__ col,
                                          const float* __restrict__ x, float lam, int v) {
  const int b = row[v], e = row[v + 1];
  const float3 xv = load3(x + 3 * v);
  float3 sum = mk(0.f, 0.f, 0.f);
  for (int k = b; k < e; ++k) sum = sum + load3(x + 3 * col[k]);
  return xv + (xv * (float)(e - b) - sum) * lam;
}

__device__ __forceinline__ void store3(float* p, float3 v) {
  p[0] = v.x;
  p[1] = v.y;
  p[2] = v.z;
}

// one atomic per CTA for each of three column sums (a warp-level atomic on
// three addresses from every warp of a large mesh serialises); called by
// every thread of the CTA after its loop
__device__ __forceinline__ void block_add3(float* dst, float3 v) {
  __shared__ float part[3][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = mk(warp_sum(v.x), warp_sum(v.y), warp_sum(v.z));
  if (lane == 0) {
    part[0][wid] = v.x;
    part[1][wid] = v.y;
    part[2][wid] = v.z;
  }
  __syncthreads();
  if (wid == 0) {
    float3 t = lane < nw ? mk(part[0][lane], part[1][lane], part[2][lane]) : mk(0.f, 0.f, 0.f);
    t = mk(warp_sum(t.x), warp_sum(t.y), warp_sum(t.z));
    if (lane == 0) {
      atomicAdd(dst, t.x);
      atomicAdd(dst + 1, t.y);
      atomicAdd(dst + 2, t.z);
    }
  }
}

// CG scratch: r, z, p, Ap as [nv][3], then scalars rz[iters + 1][3] and
// pAp[iters][3]
struct CgView {
  float *r, *z, *p, *ap, *rz, *pap;
};

__device__ __forceinline__ float safe_div(float a, float b) { return b != 0.0f ? a / b : 0.0f; }

// A column has converged once its preconditioned residual r.z has fallen
// by kCgTol2 (the residual by 1e-6) from the start: from then on its
// iterations change nothing (FP32 conjugate gradients run on in the
// rounding noise would drift).
constexpr float kCgTol2 = 1e-12f;
__device__ __forceinline__ bool cg_live(const float* rz, int it, int c) {
  return rz[3 * it + c] > kCgTol2 * rz[c];
}
__device__ __forceinline__ float cg_alpha(const CgView& v, int it, int c) {
  const float pap = v.pap[3 * it + c];
  return cg_live(v.rz, it, c) && pap > 0.0f ? v.rz[3 * it + c] / pap : 0.0f;
}


static size_t cg_bytes(int32_t nv, int32_t iters) {
  return 4 * align_up((size_t)nv * 3 * sizeof(float), 256) +
         align_up(((size_t)iters * 2 + 1) * 3 * sizeof(float), 256);
}

static CgView cg_view(void* base, int32_t nv, int32_t iters) {
  char* b = (char*)base;
  const size_t vec = align_up((size_t)nv * 3 * sizeof(float), 256);
  CgView c;
  c.r = (float*)b;
  c.z = (float*)(b + vec);
  c.p = (float*)(b + 2 * vec);
  c.ap = (float*)(b + 3 * vec);
  c.rz = (float*)(b + 4 * vec);
  c.pap = c.rz + 3 * ((size_t)iters + 1);
  return c;
}

// r = b - M x, z = r / diag, p = z, rz[0] = r . z
__global__ void k_cg_init(const int32_t* __restrict__ row, const int32_t* __restrict__ col, int32_t nv, float lam,
                          const float* __restrict__ b, const float* __restrict__ x, CgView c) {
  float3 acc = mk(0.f, 0.f, 0.f);
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x) {
    const float3 r = load3(b + 3 * v) - apply_m(row, col, x, lam, v);
    const float3 z = r * (1.0f / (1.0f + lam * (float)(row[v + 1] - row[v])));
    store3(c.r + 3 * v, r);
    store3(c.z + 3 * v, z);
    store3(c.p + 3 * v, z);
    acc = acc + mul(r, z);
  }
  block_add3(c.rz, acc);
}

// Ap = M p, pAp[it] = p . Ap
__global__ void k_cg_ap(const int32_t* __restrict__ row, const int32_t* __restrict__ col, int32_t nv, float lam,
                        CgView c, int it) {
  float3 acc = mk(0.f, 0.f, 0.f);
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x) {
    const float3 ap = apply_m(row, col, c.p, lam, v);
    store3(c.ap + 3 * v, ap);
    acc = acc + mul(load3(c.p + 3 * v), ap);
  }
  block_add3(c.pap + 3 * it, acc);
}

// alpha = rz[it] / pAp[it]; x += alpha p; r -= alpha Ap; z = r / diag;
// rz[it + 1] = r . z
__global__ void k_cg_step(const int32_t* __restrict__ row, int32_t nv, float lam, float* __restrict__ x, CgView c,
                          int it) {
  const float3 alpha = mk(cg_alpha(c, it, 0), cg_alpha(c, it, 1), cg_alpha(c, it, 2));
  float3 acc = mk(0.f, 0.f, 0.f);
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x) {
    store3(x + 3 * v, load3(x + 3 * v) + mul(alpha, load3(c.p + 3 * v)));
    const float3 r = load3(c.r + 3 * v) - mul(alpha, load3(c.ap + 3 * v));
    const float3 z = r * (1.0f / (1.0f + lam * (float)(row[v + 1] - row[v])));
    store3(c.r + 3 * v, r);
    store3(c.z + 3 * v, z);
    acc = acc + mul(r, z);
  }
  block_add3(c.rz + 3 * (it + 1), acc);
}

// beta = rz[it + 1] / rz[it]; p = z + beta p
__global__ void k_cg_dir(int32_t nv, CgView c, int it) {
  // a converged column keeps its direction at zero
  const float3 beta = mk(cg_live(c.rz, it + 1, 0) ? safe_div(c.rz[3 * (it + 1)], c.rz[3 * it]) : 0.0f,
                         cg_live(c.rz, it + 1, 1) ? safe_div(c.rz[3 * (it + 1) + 1], c.rz[3 * it + 1]) : 0.0f,
                         cg_live(c.rz, it + 1, 2) ? safe_div(c.rz[3 * (it + 1) + 2], c.rz[3 * it + 2]) : 0.0f);
  const float3 keep = mk(cg_live(c.rz, it + 1, 0) ? 1.0f : 0.0f, cg_live(c.rz, it + 1, 1) ? 1.0f : 0.0f,
                         cg_live(c.rz, it + 1, 2) ? 1.0f : 0.0f);
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x)
    store3(c.p + 3 * v, mul(keep, load3(c.z + 3 * v)) + mul(beta, load3(c.p + 3 * v)));
}

// M x = b, x holding the start on entry
static void launch_cg(const TopoView& T, int32_t nv, float lam, const float* b, float* x, int iters, void* scratch,
                      cudaStream_t s) {
  CgView c = cg_view(scratch, nv, iters);
  cudaMemsetAsync(c.rz, 0, ((size_t)iters * 2 + 1) * 3 * sizeof(float), s);
  const int g = blocks_for(nv, 256);
  k_cg_init<<<g, 256, 0, s>>>(T.row, T.col, nv, lam, b, x, c);
  for (int it = 0; it < iters; ++it) {
    k_cg_ap<<<g, 256, 0, s>>>(T.row, T.col, nv, lam, c, it);
    k_cg_step<<<g, 256, 0, s>>>(T.row, nv, lam, x, c, it);
    if (it + 1 < iters) k_cg_dir<<<g, 256, 0, s>>>(nv, c, it);
  }
}

size_t smooth_scratch_bytes(int32_t nv, int32_t iters) { return cg_bytes(nv, iters); }

void launch_smooth_solve(const void* topo, int32_t nv, int32_t nf, float lam, const float* b, float* x, int iters,
                         void* scratch, cudaStream_t s) {
  TopoView T = topo_view(const_cast<void*>(topo), nv, nf);
  ProfScope ps("smooth_solve", s);
  launch_cg(T, nv, lam, b, x, iters, scratch, s);
}

// ---------------------------------------------------------------------------
// large-steps update with AdamUniform
// ---------------------------------------------------------------------------
// optimiser state (caller-owned, zero = fresh): m [nv][3], then the step
// count and the shared second moment
struct AdamScalars {
  float v;
  int32_t t;
  float max_g2;  // scratch: max g^2 of the current step
  float pad;
};

static size_t adam_state_bytes(int32_t nv) {
  return align_up((size_t)nv * 3 * sizeof(float), 256) + sizeof(AdamScalars);
}
size_t large_steps_state_bytes(int32_t nv) { return adam_state_bytes(nv); }
size_t large_steps_scratch_bytes(int32_t nv, int32_t iters) {
  return 2 * align_up((size_t)nv * 3 * sizeof(float), 256) + cg_bytes(nv, iters);
}

__global__ void k_apply_m(const int32_t* __restrict__ row, const int32_t* __restrict__ col, int32_t nv, float lam,
                          const float* __restrict__ x, float* __restrict__ y) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x)
    store3(y + 3 * v, apply_m(row, col, x, lam, v));
}

// max g^2 over every coordinate (non-negative floats order like their bits)
__global__ void k_max_sq(const float* __restrict__ g, int64_t n, AdamScalars* sc) {
  float mx = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    mx = fmaxf(mx, g[i] * g[i]);
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, o));
  __shared__ float part[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) part[wid] = mx;
  __syncthreads();
  if (wid == 0) {  // one atomic per CTA
    mx = lane < (int)((blockDim.x + 31) >> 5) ? part[lane] : 0.f;
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, o));
    if (lane == 0) atomicMax(reinterpret_cast<int*>(&sc->max_g2), __float_as_int(mx));
  }
}

// m = b1 m + (1 - b1) g; v = b2 v + (1 - b2) max g^2 (one thread does v);
// u -= lr m_hat / (sqrt(v_hat) + eps)
__global__ void k_adam_uniform(int64_t n, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ u,
                               const AdamScalars* __restrict__ sc, float lr, float b1, float b2, float eps) {
  const int t = sc->t + 1;
  const float v = b2 * sc->v + (1.0f - b2) * sc->max_g2;
  const float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
  const float denom = sqrtf(v / c2) + eps;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float mi = b1 * m[i] + (1.0f - b1) * g[i];
    m[i] = mi;
    u[i] -= lr * (mi / c1) / denom;
  }
}

__global__ void k_adam_scalars(AdamScalars* sc, float b2) {
  sc->v = b2 * sc->v + (1.0f - b2) * sc->max_g2;
  sc->t += 1;
  sc->max_g2 = 0.f;
}

void launch_large_steps_update(const void* topo, int32_t nv, int32_t nf, float lam, float lr, float b1, float b2,
                               float eps, int iters, float* V, const float* grad, void* state, void* scratch,
                               cudaStream_t s) {
  TopoView T = topo_view(const_cast<void*>(topo), nv, nf);
  ProfScope ps("large_steps_update", s);
  const size_t vec = align_up((size_t)nv * 3 * sizeof(float), 256);
  float* u = (float*)scratch;
  float* gu = (float*)((char*)scratch + vec);
  void* cg = (char*)scratch + 2 * vec;
  float* m = (float*)state;
  AdamScalars* sc = (AdamScalars*)((char*)state + vec);
  const int g = blocks_for(nv, 256);
  const int64_t n = 3 * (int64_t)nv;
  k_apply_m<<<g, 256, 0, s>>>(T.row, T.col, nv, lam, V, u);  // u = M V
  cudaMemsetAsync(gu, 0, (size_t)n * sizeof(float), s);
  launch_cg(T, nv, lam, grad, gu, iters, cg, s);              // g_u = M^-1 dJ/dV
  k_max_sq<<<g, 256, 0, s>>>(gu, n, sc);
  k_adam_uniform<<<g, 256, 0, s>>>(n, gu, m, u, sc, lr, b1, b2, eps);
  k_adam_scalars<<<1, 1, 0, s>>>(sc, b2);
  launch_cg(T, nv, lam, u, V, iters, cg, s);                  // V = M^-1 u, from the old V
}

// ---------------------------------------------------------------------------
// L_edge
// ---------------------------------------------------------------------------
// loss[0] += sum over edges (1 - n_i . n_j)^2 / |E|; dn (unit-normal
// gradient) accumulated per vertex
__global__ void k_edge_loss(const int32_t* __restrict__ row, const int32_t* __restrict__ col, const TopoHeader* hdr,
                            int32_t nv, const float* __restrict__ N, float* __restrict__ dn,
                            float* __restrict__ loss) {
  const float inv_e = 2.0f / (float)max(hdr->nnz, 1);  // |E| = nnz / 2
  float acc = 0.f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ((nv + 31) & ~31); i += gridDim.x * blockDim.x) {
    if (i < nv) {
      const float3 ni = normalize(load3(N + 3 * i));
      float3 di = mk(0.f, 0.f, 0.f);
      for (int k = row[i]; k < row[i + 1]; ++k) {
        const int j = col[k];
        if (j <= i) continue;  // each edge once, from its smaller end
        const float3 nj = normalize(load3(N + 3 * j));
        const float e = 1.0f - dot(ni, nj);
        acc += e * e;
        const float w = -2.0f * e * inv_e;
        di = di + nj * w;
        atomicAdd(dn + 3 * j, ni.x * w);
        atomicAdd(dn + 3 * j + 1, ni.y * w);
        atomicAdd(dn + 3 * j + 2, ni.z * w);
      }
      atomicAdd(dn + 3 * i, di.x);
      atomicAdd(dn + 3 * i + 1, di.y);
      atomicAdd(dn + 3 * i + 2, di.z);
    }
    const float s = warp_sum(acc);
    acc = 0.f;
    if ((threadIdx.x & 31) == 0 && s != 0.f) atomicAdd(loss, s * inv_e);
  }
}

// dL/dN from dL/dn through n = N / |N|
__global__ void k_unit_normal_backward(int32_t nv, const float* __restrict__ N, float* __restrict__ d) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += gridDim.x * blockDim.x) {
    const float3 Nv = load3(N + 3 * i);
    const float l = len(Nv);
    const float3 n = Nv * (1.0f / l), dn = load3(d + 3 * i);
    store3(d + 3 * i, (dn - n * dot(n, dn)) * (1.0f / l));
  }
}

void launch_edge_loss_grad(const void* topo, int32_t nv, int32_t nf, const float* N, float* dN, float* loss,
                           cudaStream_t s) {
  TopoView T = topo_view(const_cast<void*>(topo), nv, nf);
  ProfScope ps("edge_loss", s);
  cudaMemsetAsync(loss, 0, sizeof(float), s);
  cudaMemsetAsync(dN, 0, (size_t)nv * 3 * sizeof(float), s);
  const int g = blocks_for(nv, 256);
  k_edge_loss<<<g, 256, 0, s>>>(T.row, T.col, T.hdr, nv, N, dN, loss);
  k_unit_normal_backward<<<g, 256, 0, s>>>(nv, N, dN);
}

// device pointers of the CSR arrays
void topology_csr(const void* topo, int32_t nv, int32_t nf, const int32_t** row, const int32_t** col) {
  const TopoView T = topo_view(const_cast<void*>(topo), nv, nf);
  *row = T.row;
  *col = T.col;
}

// host copy of the header (n edges etc.), for the binding
void read_topology_header(const void* topo, int32_t* nnz, int32_t* max_deg, cudaStream_t s) {
  TopoHeader h;
  cudaMemcpyAsync(&h, topo, sizeof(h), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  *nnz = h.nnz;
  *max_deg = h.max_deg;
}

}  // namespace dt

// C ABI of libdifftrans (declared in include/difftrans.h): argument checks on
// the host, then stream-ordered launches.  No device memory is allocated
// here; every buffer comes from the caller.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include <string.h>

#include "dt_internal.cuh"

namespace dt {

// implemented in the other translation units
void launch_vertex_normals(const float* V, int32_t nv, const int32_t* F, int32_t nf, float* N, void* scratch,
                           cudaStream_t s);
size_t normals_scratch_bytes(int32_t nv);
void launch_vertex_normals_backward(const float* V, int32_t nv, const int32_t* F, int32_t nf, const float* dN,
                                    float* dV, cudaStream_t s);
size_t bvh_scratch_bytes(int32_t nf);
void launch_build(const float* V, const int32_t* F, int32_t nf, void* bvh, void* scratch, cudaStream_t s);
void launch_refit(const float* V, const int32_t* F, int32_t nf, void* bvh, void* scratch, cudaStream_t s);
SceneEntry make_entry(const dt_scene& sc, const dt_views& vw, const dt_params& p, float* out);
void finish_table(SceneEntry* entries, int n, TableHeader& th);
void launch_forward_table(const TableHeader& th, const SceneEntry* entries, void* ws, unsigned long long cap,
                          unsigned long long ring, bool mom, cudaStream_t s);
void launch_backward_table(const TableHeader& th, const SceneEntry* entries, const void* ws, unsigned long long cap,
                           unsigned long long ring, bool mom, void* bws, unsigned long long max_level, cudaStream_t s);
size_t backward_ws_bytes_table(unsigned long long max_level, const SceneEntry* entries, int n);
void assign_dN(SceneEntry* entries, int n, void* bws, unsigned long long max_level);
void launch_dump(const void* ws, unsigned long long cap, int32_t* si, float* sf, unsigned long long n,
                 cudaStream_t s);
void launch_closest_hit(const void* bvh, int32_t nf, const float* o, const float* d, const int32_t* src, int32_t n,
                        float tmin, int32_t* tri, float* tbb, cudaStream_t s);
void launch_paper_loss_grad(const float* img, const float* target, int64_t n, float lc, float lt, float* grad,
                            float* loss, cudaStream_t s);
void launch_l2_loss_grad(const float* img, const float* target, int64_t n, float scale, float* grad, float* loss,
                         cudaStream_t s);
size_t topology_bytes(int32_t nv, int32_t nf);
void launch_build_topology(const int32_t* F, int32_t nf, int32_t nv, void* topo, cudaStream_t s);
void read_topology_header(const void* topo, int32_t* nnz, int32_t* max_deg, cudaStream_t s);
void topology_csr(const void* topo, int32_t nv, int32_t nf, const int32_t** row, const int32_t** col);
size_t smooth_scratch_bytes(int32_t nv, int32_t iters);
void launch_smooth_solve(const void* topo, int32_t nv, int32_t nf, float lam, const float* b, float* x, int iters,
                         void* scratch, cudaStream_t s);
size_t large_steps_state_bytes(int32_t nv);
size_t large_steps_scratch_bytes(int32_t nv, int32_t iters);
void launch_large_steps_update(const void* topo, int32_t nv, int32_t nf, float lam, float lr, float b1, float b2,
                               float eps, int iters, float* V, const float* grad, void* state, void* scratch,
                               cudaStream_t s);
void launch_edge_loss_grad(const void* topo, int32_t nv, int32_t nf, const float* N, float* dN, float* loss,
                           cudaStream_t s);

// Launch and scheduling knobs (dt_set_tuning); process-wide.  Node visits
// per scheduling round 192, refill at 8 idle lanes, 5 traversal and 4
// shading CTAs per SM, binary nodes, binned SAH builder, levels after the
// camera rays traced in the order of 20-bit buckets.
dt_tuning g_tuning = {192, 8, 5, 4, 2, 1, 20, 65536};

static thread_local char g_err[512] = "";

dt_status set_error(dt_status code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

dt_status check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(DT_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
  g_err[0] = 0;
  return DT_OK;
}

int num_sms() {
  static std::mutex mu;
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  std::lock_guard<std::mutex> lk(mu);
  if (!cache[dev]) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
    cache[dev] = n;
  }
  return cache[dev];
}

static bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

// ---- per-kernel CUDA-event timing ------------------------------------------
namespace {
struct ProfRec {
  std::string name;
  cudaEvent_t start, stop;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRec> g_prof;
std::vector<cudaEvent_t> g_prof_pool;

cudaEvent_t prof_event() {
  if (!g_prof_pool.empty()) {
    cudaEvent_t e = g_prof_pool.back();
    g_prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
}  // namespace

ProfScope::ProfScope(const char* name, cudaStream_t s) : slot(-1), stream(s) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (!g_prof_on) return;
  ProfRec r{name, prof_event(), prof_event()};
  cudaEventRecord(r.start, s);
  g_prof.push_back(r);
  slot = (int)g_prof.size() - 1;
}

ProfScope::~ProfScope() {
  if (slot < 0) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (slot < (int)g_prof.size()) cudaEventRecord(g_prof[slot].stop, stream);
}

// the largest segment capacity whose layout fits in ws_bytes, with a hit ring
// of `ring` records per level parity (ring = 0: one hit record per segment)
// and, for tape_mode 2, the medium moments of every segment
static unsigned long long cap_from_bytes(size_t ws_bytes, unsigned long long ring = 0, bool mom = false) {
  const size_t fixed = 1024 + kTableBytes + kOrderBytes + 4096 + (ring ? 2 * ring * 16 : 0);
  if (ws_bytes < fixed) return 0;
  unsigned long long cap = (ws_bytes - fixed + 4096) / ((ring ? 56 : 72) + (mom ? 4 * kMomFloats : 0));
  if (cap > 0x7fffffffull) cap = 0x7fffffffull;
  while (cap > 0 && WsLayout(cap, ring, mom).total > ws_bytes) --cap;
  return cap;
}

static dt_status check_scene(const dt_scene* sc) {
  if (!sc) return set_error(DT_ERR_INVALID_ARG, "scene is NULL");
  if (!sc->d_V || !sc->d_F || !sc->d_bvh || !sc->d_N || !sc->d_ior || !sc->d_sigma || !sc->d_env)
    return set_error(DT_ERR_INVALID_ARG, "scene has a NULL device pointer");
  if (sc->nv < 3 || sc->nf < 1) return set_error(DT_ERR_INVALID_ARG, "scene needs nv >= 3 and nf >= 1 (nv=%d nf=%d)",
                                                 sc->nv, sc->nf);
  if (sc->env_w < 1 || sc->env_h < 1) return set_error(DT_ERR_INVALID_ARG, "environment size must be positive");
  if (!aligned(sc->d_bvh, 256)) return set_error(DT_ERR_INVALID_ARG, "BVH buffer must be 256-byte aligned");
  if (sc->medium) {
    const dt_medium& M = *sc->medium;
    if (!M.d_mu || !aligned(M.d_mu, 16) || (M.d_grad_mu && !aligned(M.d_grad_mu, 16)))
      return set_error(DT_ERR_INVALID_ARG, "medium node values (and gradient) need 16-byte aligned device pointers");
    if (M.levels < 0 || M.levels > DT_MAX_HASH_LEVELS)
      return set_error(DT_ERR_INVALID_ARG, "medium levels must be 0 (dense grid) or 1..%d (got %d)",
                       DT_MAX_HASH_LEVELS, M.levels);
    if (M.levels == 0) {
      if (M.nx < 2 || M.ny < 2 || M.nz < 2 || (long long)M.nx * M.ny * M.nz > (1ll << 31))
        return set_error(DT_ERR_INVALID_ARG, "medium needs at least 2 nodes per axis (got %d x %d x %d)", M.nx, M.ny,
                         M.nz);
    } else {
      if (M.log2_table < 4 || M.log2_table > 24)
        return set_error(DT_ERR_INVALID_ARG, "hash texture log2_table must be in 4..24 (got %d)", M.log2_table);
      for (int l = 0; l < M.levels; ++l)
        if (M.res[l] < 2 || M.res[l] > (1 << 20))
          return set_error(DT_ERR_INVALID_ARG, "hash texture level %d needs 2..2^20 nodes per axis (got %d)", l,
                           M.res[l]);
    }
    for (int a = 0; a < 3; ++a)
      if (!(M.hi[a] > M.lo[a]) || !std::isfinite(M.hi[a] - M.lo[a]))
        return set_error(DT_ERR_INVALID_ARG, "medium box needs hi > lo on every axis");
    if (!(M.step > 0.0f) || !std::isfinite(M.step)) return set_error(DT_ERR_INVALID_ARG, "medium step must be > 0");
  }
  return DT_OK;
}

static dt_status check_views_params(const dt_views* vw, const dt_params* p) {
  if (!vw || !p) return set_error(DT_ERR_INVALID_ARG, "views or params is NULL");
  if (!vw->d_cams) return set_error(DT_ERR_INVALID_ARG, "views.d_cams is NULL");
  if (vw->n_views < 1 || vw->width < 1 || vw->height < 1)
    return set_error(DT_ERR_INVALID_ARG, "views need n_views, width, height >= 1");
  if (p->max_depth < 0 || p->max_depth > kMaxDepth)
    return set_error(DT_ERR_INVALID_ARG, "max_depth must be in [0, %d] (got %d)", kMaxDepth, p->max_depth);
  if (p->spp < 1) return set_error(DT_ERR_INVALID_ARG, "spp must be >= 1");
  if (!(p->t_min >= 0.0f)) return set_error(DT_ERR_INVALID_ARG, "t_min must be >= 0");
  if (p->tape_mode < 0 || p->tape_mode > 2) return set_error(DT_ERR_INVALID_ARG, "tape_mode must be 0, 1 or 2");
  if (p->tape_mode == 1 && p->level_capacity < 1)
    return set_error(DT_ERR_INVALID_ARG, "tape_mode 1 needs level_capacity >= 1");
  const unsigned long long n0 = (unsigned long long)vw->n_views * vw->width * vw->height * p->spp;
  if (n0 >= 0xffffffffull) return set_error(DT_ERR_INVALID_ARG, "too many primary rays in one call (%llu)", n0);
  return DT_OK;
}

}  // namespace dt

using namespace dt;

extern "C" {

const char* dt_last_error(void) { return g_err; }
const char* dt_version(void) { return "difftrans-gb300 0.3 (sm_103a)"; }

dt_status dt_vertex_normals_scratch_size(int32_t nv, size_t* bytes) {
  if (nv < 1 || !bytes) return set_error(DT_ERR_INVALID_ARG, "need nv >= 1 and a size pointer");
  *bytes = normals_scratch_bytes(nv);
  return DT_OK;
}

dt_status dt_vertex_normals(const float* d_V, int32_t nv, const int32_t* d_F, int32_t nf, float* d_N,
                            void* d_scratch, dt_stream stream) {
  if (!d_V || !d_F || !d_N || !d_scratch) return set_error(DT_ERR_INVALID_ARG, "NULL pointer");
  if (nv < 1 || nf < 1) return set_error(DT_ERR_INVALID_ARG, "nv and nf must be >= 1");
  if (!aligned(d_scratch, 8)) return set_error(DT_ERR_INVALID_ARG, "scratch must be 8-byte aligned");
  launch_vertex_normals(d_V, nv, d_F, nf, d_N, d_scratch, (cudaStream_t)stream);
  return check_launch("dt_vertex_normals");
}

dt_status dt_vertex_normals_backward(const float* d_V, int32_t nv, const int32_t* d_F, int32_t nf, const float* d_dN,
                                     float* d_dV, dt_stream stream) {
  if (!d_V || !d_F || !d_dN || !d_dV) return set_error(DT_ERR_INVALID_ARG, "NULL pointer");
  if (nv < 1 || nf < 1) return set_error(DT_ERR_INVALID_ARG, "nv and nf must be >= 1");
  launch_vertex_normals_backward(d_V, nv, d_F, nf, d_dN, d_dV, (cudaStream_t)stream);
  return check_launch("dt_vertex_normals_backward");
}

dt_status dt_bvh_size(int32_t nf, size_t* bvh_bytes, size_t* scratch_bytes) {
  if (nf < 1) return set_error(DT_ERR_INVALID_ARG, "nf must be >= 1");
  if (nf > (1 << 30)) return set_error(DT_ERR_INVALID_ARG, "nf must be <= 2^30");
  if (bvh_bytes) *bvh_bytes = BvhLayout(nf).total;
  if (scratch_bytes) *scratch_bytes = bvh_scratch_bytes(nf);
  return DT_OK;
}

dt_status dt_build_bvh(const float* d_V, int32_t nv, const int32_t* d_F, int32_t nf, void* d_bvh, void* d_scratch,
                       dt_stream stream) {
  if (!d_V || !d_F || !d_bvh || !d_scratch) return set_error(DT_ERR_INVALID_ARG, "NULL pointer");
  if (nv < 3 || nf < 1 || nf > (1 << 30)) return set_error(DT_ERR_INVALID_ARG, "need nv >= 3 and 1 <= nf <= 2^30");
  if (!aligned(d_bvh, 256) || !aligned(d_scratch, 256))
    return set_error(DT_ERR_INVALID_ARG, "BVH and scratch buffers must be 256-byte aligned");
  launch_build(d_V, d_F, nf, d_bvh, d_scratch, (cudaStream_t)stream);
  return check_launch("dt_build_bvh");
}

dt_status dt_refit_bvh(const float* d_V, int32_t nv, const int32_t* d_F, int32_t nf, void* d_bvh, void* d_scratch,
                       dt_stream stream) {
  if (!d_V || !d_F || !d_bvh || !d_scratch) return set_error(DT_ERR_INVALID_ARG, "NULL pointer");
  if (nv < 3 || nf < 1 || nf > (1 << 30)) return set_error(DT_ERR_INVALID_ARG, "need nv >= 3 and 1 <= nf <= 2^30");
  if (!aligned(d_bvh, 256) || !aligned(d_scratch, 256))
    return set_error(DT_ERR_INVALID_ARG, "BVH and scratch buffers must be 256-byte aligned");
  launch_refit(d_V, d_F, nf, d_bvh, d_scratch, (cudaStream_t)stream);
  return check_launch("dt_refit_bvh");
}

dt_status dt_render_workspace_size(int64_t seg_capacity, size_t* ws_bytes) {
  if (seg_capacity < 1 || seg_capacity > 0x7fffffffll)
    return set_error(DT_ERR_INVALID_ARG, "seg_capacity must be in [1, 2^31-1]");
  if (!ws_bytes) return set_error(DT_ERR_INVALID_ARG, "ws_bytes is NULL");
  *ws_bytes = WsLayout((unsigned long long)seg_capacity).total;
  return DT_OK;
}

dt_status dt_render_workspace_size_ex(int64_t seg_capacity, int32_t tape_mode, int64_t level_capacity,
                                      size_t* ws_bytes) {
  if (seg_capacity < 1 || seg_capacity > 0x7fffffffll)
    return set_error(DT_ERR_INVALID_ARG, "seg_capacity must be in [1, 2^31-1]");
  if (!ws_bytes) return set_error(DT_ERR_INVALID_ARG, "ws_bytes is NULL");
  if (tape_mode == 0 || tape_mode == 2) {
    *ws_bytes = WsLayout((unsigned long long)seg_capacity, 0, tape_mode == 2).total;
    return DT_OK;
  }
  if (tape_mode != 1 || level_capacity < 1 || level_capacity > seg_capacity)
    return set_error(DT_ERR_INVALID_ARG, "tape_mode must be 0, 1 or 2, and tape_mode 1 needs 1 <= level_capacity "
                                         "<= seg_capacity");
  *ws_bytes = WsLayout((unsigned long long)seg_capacity, (unsigned long long)level_capacity).total;
  return DT_OK;
}

dt_status dt_render(const dt_scene* scene, const dt_views* views, const dt_params* params, float* d_out, void* d_ws,
                    size_t ws_bytes, dt_stream stream) {
  if (!scene || !views || !params) return set_error(DT_ERR_INVALID_ARG, "scene, views or params is NULL");
  dt_batch_entry e;
  memset(&e, 0, sizeof(e));
  e.scene = *scene;
  e.views = *views;
  e.params = *params;
  e.d_out = d_out;
  return dt_render_batch(&e, 1, d_ws, ws_bytes, stream);
}

static dt_status check_entries(const dt_batch_entry* entries, int32_t n, bool backward,
                               std::vector<SceneEntry>& out, TableHeader& th) {
  if (!entries) return set_error(DT_ERR_INVALID_ARG, "entries is NULL");
  if (n < 1 || n > kMaxBatch) return set_error(DT_ERR_INVALID_ARG, "batch size must be in [1, %d] (got %d)", kMaxBatch, n);
  out.resize(n);
  unsigned long long total = 0;
  for (int i = 0; i < n; ++i) {
    const dt_batch_entry& e = entries[i];
    dt_status st = check_scene(&e.scene);
    if (st == DT_OK) st = check_views_params(&e.views, &e.params);
    if (st != DT_OK) {
      char msg[sizeof(g_err)];
      strncpy(msg, g_err, sizeof(msg) - 1);
      msg[sizeof(msg) - 1] = 0;
      return set_error(st, "entry %d: %s", i, msg);
    }
    if (!backward && !e.d_out) return set_error(DT_ERR_INVALID_ARG, "entry %d: d_out is NULL", i);
    if (backward && (!e.d_grad_out || !e.d_grad_V || !e.d_grad_ior || !e.d_grad_sigma))
      return set_error(DT_ERR_INVALID_ARG, "entry %d: a gradient pointer is NULL", i);
    out[i] = make_entry(e.scene, e.views, e.params, e.d_out);
    out[i].grad_out = e.d_grad_out;
    out[i].dV = e.d_grad_V;
    out[i].dior = e.d_grad_ior;
    out[i].dsigma = e.d_grad_sigma;
    total += (unsigned long long)out[i].pix_count * (unsigned long long)e.params.spp;
  }
  if (total >= 0xffffffffull) return set_error(DT_ERR_INVALID_ARG, "too many primary rays in one call (%llu)", total);
  for (int i = 1; i < n; ++i)
    if (entries[i].params.tape_mode != entries[0].params.tape_mode ||
        (entries[0].params.tape_mode == 1 && entries[i].params.level_capacity != entries[0].params.level_capacity))
      return set_error(DT_ERR_INVALID_ARG, "entry %d: all entries of a batch share tape_mode and level_capacity", i);
  finish_table(out.data(), n, th);
  return DT_OK;
}

static unsigned long long ring_of(const dt_batch_entry* entries) {
  return entries[0].params.tape_mode == 1 ? (unsigned long long)entries[0].params.level_capacity : 0ull;
}
static bool mom_of(const dt_batch_entry* entries) { return entries[0].params.tape_mode == 2; }

dt_status dt_render_batch(const dt_batch_entry* entries, int32_t n, void* d_ws, size_t ws_bytes, dt_stream stream) {
  std::vector<SceneEntry> ent;
  TableHeader th;
  dt_status st = check_entries(entries, n, false, ent, th);
  if (st) return st;
  if (!d_ws) return set_error(DT_ERR_INVALID_ARG, "workspace is NULL");
  if (!aligned(d_ws, 256)) return set_error(DT_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  const unsigned long long ring = ring_of(entries);
  const bool mom = mom_of(entries);
  const unsigned long long cap = cap_from_bytes(ws_bytes, ring, mom);
  if (cap < th.n_samples)
    return set_error(DT_ERR_INVALID_ARG, "workspace holds %llu segments, fewer than the %u camera rays", cap,
                     th.n_samples);
  launch_forward_table(th, ent.data(), d_ws, cap, ring, mom, (cudaStream_t)stream);
  return check_launch("dt_render");
}

dt_status dt_read_stats(const void* d_ws, size_t ws_bytes, dt_stats* out, dt_stream stream) {
  if (!d_ws || !out) return set_error(DT_ERR_INVALID_ARG, "NULL pointer");
  if (cap_from_bytes(ws_bytes) == 0) return set_error(DT_ERR_INVALID_ARG, "workspace too small");
  WsHeader h;
  cudaError_t e = cudaMemcpyAsync(&h, d_ws, sizeof(WsHeader), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return set_error(DT_ERR_CUDA, "dt_read_stats: %s", cudaGetErrorString(e));
  memset(out, 0, sizeof(*out));
  out->status = (h.status & ST_QUEUE_OVERFLOW) ? DT_ERR_QUEUE_OVERFLOW
              : (h.status & ST_STACK_OVERFLOW) ? DT_ERR_STACK_OVERFLOW : DT_OK;
  out->n_levels = (int32_t)h.n_levels;
  long long seg = 0, need = 0, mx = 0, lvl_need = 0;
  for (int k = 0; k < kMaxLevels; ++k) {
    const unsigned long long start = h.level_start[k];
    unsigned long long n = h.level_count[k];
    need += (long long)n;
    if ((long long)n > lvl_need) lvl_need = (long long)n;
    if (h.ring && n > h.ring) n = h.ring;
    if (k >= (int)h.n_levels) n = 0;
    const unsigned long long room = start < h.capacity ? h.capacity - start : 0ull;
    if (n > room) n = room;
    out->level_count[k] = (int64_t)n;
    out->level_start[k] = (int64_t)start;
    seg += (long long)n;
    if ((long long)n > mx) mx = (long long)n;
  }
  out->segments = seg;
  out->seg_needed = need;
  out->max_level = mx;
  out->level_needed = lvl_need;
  if (h.ring && lvl_need > (long long)h.ring && out->status == DT_OK) out->status = DT_ERR_QUEUE_OVERFLOW;
  out->hits = (int64_t)h.counters[CNT_HITS];
  out->misses = (int64_t)h.counters[CNT_MISSES];
  out->discarded = (int64_t)h.counters[CNT_DISCARDED];
  out->backfacing = (int64_t)h.counters[CNT_BACKFACING];
  out->tir = (int64_t)h.counters[CNT_TIR];
  out->nodes_visited = (int64_t)h.counters[CNT_NODES];
  out->tris_tested = (int64_t)h.counters[CNT_TRIS];
  out->medium_samples = (int64_t)h.counters[CNT_MEDIUM];
  g_err[0] = 0;
  return DT_OK;
}

dt_status dt_backward_workspace_size(int64_t max_level, int32_t nv, size_t* bytes) {
  if (max_level < 1 || nv < 1 || !bytes) return set_error(DT_ERR_INVALID_ARG, "need max_level >= 1, nv >= 1");
  SceneEntry e;
  memset(&e, 0, sizeof(e));
  e.nv = nv;
  *bytes = backward_ws_bytes_table((unsigned long long)max_level, &e, 1);
  return DT_OK;
}

dt_status dt_batch_backward_workspace_size(const dt_batch_entry* entries, int32_t n, int64_t max_level,
                                           size_t* bytes) {
  if (!entries || n < 1 || n > kMaxBatch || max_level < 1 || !bytes) return set_error(DT_ERR_INVALID_ARG, "bad argument");
  std::vector<SceneEntry> e(n);
  for (int i = 0; i < n; ++i) {
    memset(&e[i], 0, sizeof(SceneEntry));
    e[i].nv = entries[i].scene.nv;
  }
  *bytes = backward_ws_bytes_table((unsigned long long)max_level, e.data(), n);
  return DT_OK;
}

dt_status dt_render_batch_backward(const dt_batch_entry* entries, int32_t n, const void* d_ws, size_t ws_bytes,
                                   void* d_bws, size_t bws_bytes, int64_t max_level, dt_stream stream) {
  std::vector<SceneEntry> ent;
  TableHeader th;
  dt_status st = check_entries(entries, n, true, ent, th);
  if (st) return st;
  if (!d_ws || !d_bws) return set_error(DT_ERR_INVALID_ARG, "NULL workspace");
  const unsigned long long ring = ring_of(entries);
  const bool mom = mom_of(entries);
  const unsigned long long cap = cap_from_bytes(ws_bytes, ring, mom);
  if (cap == 0) return set_error(DT_ERR_INVALID_ARG, "workspace too small");
  if (max_level < 1) return set_error(DT_ERR_INVALID_ARG, "max_level must be >= 1");
  if (bws_bytes < backward_ws_bytes_table((unsigned long long)max_level, ent.data(), n))
    return set_error(DT_ERR_INVALID_ARG, "backward workspace smaller than its size query");
  if (!aligned(d_bws, 256)) return set_error(DT_ERR_INVALID_ARG, "backward workspace must be 256-byte aligned");
  assign_dN(ent.data(), n, d_bws, (unsigned long long)max_level);
  launch_backward_table(th, ent.data(), d_ws, cap, ring, mom, d_bws, (unsigned long long)max_level,
                        (cudaStream_t)stream);
  return check_launch("dt_render_backward");
}

dt_status dt_render_backward(const dt_scene* scene, const dt_views* views, const dt_params* params, const void* d_ws,
                             size_t ws_bytes, const float* d_grad_out, float* d_grad_V, float* d_grad_ior,
                             float* d_grad_sigma, void* d_bws, size_t bws_bytes, int64_t max_level,
                             dt_stream stream) {
  if (!scene || !views || !params) return set_error(DT_ERR_INVALID_ARG, "scene, views or params is NULL");
  dt_batch_entry e;
  memset(&e, 0, sizeof(e));
  e.scene = *scene;
  e.views = *views;
  e.params = *params;
  e.d_grad_out = d_grad_out;
  e.d_grad_V = d_grad_V;
  e.d_grad_ior = d_grad_ior;
  e.d_grad_sigma = d_grad_sigma;
  return dt_render_batch_backward(&e, 1, d_ws, ws_bytes, d_bws, bws_bytes, max_level, stream);
}

dt_status dt_dump_segments(const void* d_ws, size_t ws_bytes, int32_t* d_seg_i, float* d_seg_f, int64_t cap,
                           dt_stream stream) {
  if (!d_ws || !d_seg_i || !d_seg_f || cap < 0) return set_error(DT_ERR_INVALID_ARG, "bad argument");
  const unsigned long long wcap = cap_from_bytes(ws_bytes, 0);
  if (wcap == 0) return set_error(DT_ERR_INVALID_ARG, "workspace too small");
  launch_dump(d_ws, wcap, d_seg_i, d_seg_f, (unsigned long long)cap, (cudaStream_t)stream);
  return check_launch("dt_dump_segments");
}

dt_status dt_get_tuning(dt_tuning* out) {
  if (!out) return set_error(DT_ERR_INVALID_ARG, "NULL pointer");
  *out = g_tuning;
  return DT_OK;
}

dt_status dt_set_tuning(const dt_tuning* in) {
  if (!in) return set_error(DT_ERR_INVALID_ARG, "NULL pointer");
  if (in->trace_steps < 1 || in->trace_steps > 256 || in->trace_refill < 1 || in->trace_refill > 32 ||
      in->trace_blocks_per_sm < 1 || in->trace_blocks_per_sm > 8 || in->shade_blocks_per_sm < 1 ||
      in->shade_blocks_per_sm > 16 || (in->bvh_width != 2 && in->bvh_width != 4) ||
      (in->bvh_builder != 0 && in->bvh_builder != 1) ||
      (in->trace_order != 0 && (in->trace_order < 12 || in->trace_order > kOrderBits)) || in->order_min_rays < 0)
    return set_error(DT_ERR_INVALID_ARG, "tuning out of range (steps 1..256, refill 1..32, trace blocks/SM 1..8, "
                                         "shade blocks/SM 1..16, width 2 or 4, builder 0 or 1, order 0 or 12..22, "
                                         "order_min_rays >= 0)");
  g_tuning = *in;
  return DT_OK;
}

dt_status dt_profile_enable(int32_t enable) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_on = enable != 0;
  return DT_OK;
}

dt_status dt_profile_read(dt_kernel_time* out, int32_t cap, int32_t* n) {
  if (!n || (cap > 0 && !out)) return set_error(DT_ERR_INVALID_ARG, "NULL pointer");
  std::lock_guard<std::mutex> lk(g_prof_mu);
  std::vector<std::string> names;
  std::vector<int64_t> cnt;
  std::vector<double> ms;
  for (ProfRec& r : g_prof) {
    cudaError_t e = cudaEventSynchronize(r.stop);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.start, r.stop);
    if (e != cudaSuccess) return set_error(DT_ERR_CUDA, "dt_profile_read: %s", cudaGetErrorString(e));
    size_t k = 0;
    while (k < names.size() && names[k] != r.name) ++k;
    if (k == names.size()) { names.push_back(r.name); cnt.push_back(0); ms.push_back(0.0); }
    cnt[k] += 1;
    ms[k] += t;
    g_prof_pool.push_back(r.start);
    g_prof_pool.push_back(r.stop);
  }
  g_prof.clear();
  *n = (int32_t)names.size();
  for (int32_t k = 0; k < *n && k < cap; ++k) {
    memset(out[k].name, 0, sizeof(out[k].name));
    strncpy(out[k].name, names[k].c_str(), sizeof(out[k].name) - 1);
    out[k].launches = cnt[k];
    out[k].total_ms = ms[k];
  }
  return DT_OK;
}

dt_status dt_l2_loss_grad(const float* d_img, const float* d_target, int64_t n, float scale, float* d_grad,
                          float* d_loss, dt_stream stream) {
  if (!d_img || !d_target || !d_grad || !d_loss || n < 0) return set_error(DT_ERR_INVALID_ARG, "bad argument");
  launch_l2_loss_grad(d_img, d_target, n, scale, d_grad, d_loss, (cudaStream_t)stream);
  return check_launch("dt_l2_loss_grad");
}


static dt_status check_mesh(int32_t nv, int32_t nf) {
  if (nv < 3 || nf < 1 || (int64_t)nf * 6 > 0x7fffffffll) return set_error(DT_ERR_INVALID_ARG, "need nv >= 3, nf >= 1");
  return DT_OK;
}

dt_status dt_topology_size(int32_t nv, int32_t nf, size_t* bytes) {
  if (!bytes) return set_error(DT_ERR_INVALID_ARG, "NULL pointer");
  if (dt_status st = check_mesh(nv, nf)) return st;
  *bytes = topology_bytes(nv, nf);
  return DT_OK;
}

dt_status dt_build_topology(const int32_t* d_F, int32_t nf, int32_t nv, void* d_topo, size_t topo_bytes,
                            dt_stream stream) {
  if (dt_status st = check_mesh(nv, nf)) return st;
  if (!d_F || !d_topo || !aligned(d_topo, 256) || topo_bytes < topology_bytes(nv, nf))
    return set_error(DT_ERR_INVALID_ARG, "bad topology buffer");
  launch_build_topology(d_F, nf, nv, d_topo, (cudaStream_t)stream);
  return check_launch("dt_build_topology");
}

dt_status dt_topology_info(const void* d_topo, int32_t nv, int32_t nf, int64_t* n_edges, int32_t* max_degree,
                           const int32_t** d_row, const int32_t** d_col, dt_stream stream) {
  if (dt_status st = check_mesh(nv, nf)) return st;
  if (!d_topo) return set_error(DT_ERR_INVALID_ARG, "NULL topology");
  int32_t nnz = 0, md = 0;
  read_topology_header(d_topo, &nnz, &md, (cudaStream_t)stream);
  if (n_edges) *n_edges = nnz / 2;
  if (max_degree) *max_degree = md;
  const int32_t *row = nullptr, *col = nullptr;
  topology_csr(d_topo, nv, nf, &row, &col);
  if (d_row) *d_row = row;
  if (d_col) *d_col = col;
  return check_launch("dt_topology_info");
}

dt_status dt_smooth_scratch_size(int32_t nv, int32_t iters, size_t* bytes) {
  if (!bytes || nv < 1 || iters < 1) return set_error(DT_ERR_INVALID_ARG, "bad argument");
  *bytes = smooth_scratch_bytes(nv, iters);
  return DT_OK;
}

dt_status dt_smooth_solve(const void* d_topo, int32_t nv, int32_t nf, float lambda, const float* d_b, float* d_x,
                          int32_t iters, void* d_scratch, size_t scratch_bytes, dt_stream stream) {
  if (dt_status st = check_mesh(nv, nf)) return st;
  if (!d_topo || !d_b || !d_x || !d_scratch || iters < 1 || iters > 100000 || !(lambda >= 0.0f) ||
      scratch_bytes < smooth_scratch_bytes(nv, iters) || !aligned(d_scratch, 256))
    return set_error(DT_ERR_INVALID_ARG, "bad argument");
  launch_smooth_solve(d_topo, nv, nf, lambda, d_b, d_x, iters, d_scratch, (cudaStream_t)stream);
  return check_launch("dt_smooth_solve");
}

dt_status dt_large_steps_sizes(int32_t nv, int32_t iters, size_t* state_bytes, size_t* scratch_bytes) {
  if (!state_bytes || !scratch_bytes || nv < 1 || iters < 1) return set_error(DT_ERR_INVALID_ARG, "bad argument");
  *state_bytes = large_steps_state_bytes(nv);
  *scratch_bytes = large_steps_scratch_bytes(nv, iters);
  return DT_OK;
}

dt_status dt_large_steps_update(const void* d_topo, int32_t nv, int32_t nf, float lambda, float lr, float beta1,
                                float beta2, float eps, int32_t iters, float* d_V, const float* d_grad_V,
                                void* d_state, void* d_scratch, size_t scratch_bytes, dt_stream stream) {
  if (dt_status st = check_mesh(nv, nf)) return st;
  if (!d_topo || !d_V || !d_grad_V || !d_state || !d_scratch || iters < 1 || iters > 100000 || !(lambda >= 0.0f) ||
      !(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f) ||
      scratch_bytes < large_steps_scratch_bytes(nv, iters) || !aligned(d_scratch, 256) || !aligned(d_state, 16))
    return set_error(DT_ERR_INVALID_ARG, "bad argument");
  launch_large_steps_update(d_topo, nv, nf, lambda, lr, beta1, beta2, eps, iters, d_V, d_grad_V, d_state, d_scratch,
                            (cudaStream_t)stream);
  return check_launch("dt_large_steps_update");
}

dt_status dt_edge_loss_grad(const void* d_topo, int32_t nv, int32_t nf, const float* d_N, float* d_grad_N,
                            float* d_loss, dt_stream stream) {
  if (dt_status st = check_mesh(nv, nf)) return st;
  if (!d_topo || !d_N || !d_grad_N || !d_loss) return set_error(DT_ERR_INVALID_ARG, "bad argument");
  launch_edge_loss_grad(d_topo, nv, nf, d_N, d_grad_N, d_loss, (cudaStream_t)stream);
  return check_launch("dt_edge_loss_grad");
}

dt_status dt_paper_loss_grad(const float* d_img, const float* d_target, int64_t n_pix, float lambda_color,
                             float lambda_tone, float* d_grad, float* d_loss, dt_stream stream) {
  if (!d_loss || n_pix < 0 || (n_pix > 0 && (!d_img || !d_target || !d_grad)))
    return set_error(DT_ERR_INVALID_ARG, "bad argument");
  launch_paper_loss_grad(d_img, d_target, n_pix, lambda_color, lambda_tone, d_grad, d_loss, (cudaStream_t)stream);
  return check_launch("dt_paper_loss_grad");
}

dt_status dt_closest_hit(const void* d_bvh, int32_t nf, const float* d_o, const float* d_d, const int32_t* d_src,
                         int32_t n, float t_min, int32_t* d_tri, float* d_tbb, dt_stream stream) {
  if (!d_bvh || !d_o || !d_d || !d_tri || !d_tbb) return set_error(DT_ERR_INVALID_ARG, "NULL pointer");
  if (nf < 1 || n < 0) return set_error(DT_ERR_INVALID_ARG, "need nf >= 1 and n >= 0");
  if (!aligned(d_bvh, 256)) return set_error(DT_ERR_INVALID_ARG, "BVH buffer must be 256-byte aligned");
  if (n == 0) return DT_OK;
  launch_closest_hit(d_bvh, nf, d_o, d_d, d_src, n, t_min, d_tri, d_tbb, (cudaStream_t)stream);
  return check_launch("dt_closest_hit");
}

}  // extern "C"

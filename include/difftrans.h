/*
 * difftrans.h -- C ABI of the GB300 (sm_103a) recursive differentiable
 * transparent-mesh ray tracer of DiffTrans (arXiv 2603.00413).
 *
 * Problem statement (Sec. 3.4, "Differentiable Mesh Intersection" and
 * "Optimization"): a closed triangle mesh M = (V, E, F) with a uniform index
 * of refraction and an absorption rate is rendered by a recursive ray tracer
 * (Sec. 3.4 "Recursive Ray Tracing", steps 1-5) whose rays split at every
 * surface hit into a Fresnel-weighted reflected and a Snell-refracted ray
 * (Sec. 3.3, Eqs. 3-8), are attenuated inside the object by Beer-Lambert
 * absorption (Eqs. 9-11), and read the environment where they escape.  The
 * backward pass returns the gradient of an image loss with respect to the
 * vertex positions, the IoR and the per-channel absorption.
 *
 * Conventions of the whole interface
 *  - Every pointer named d_* is DEVICE memory of the current CUDA device,
 *    owned by the caller; every other pointer is host memory owned by the
 *    caller.  The library allocates no device memory: each call that needs
 *    workspace takes a caller buffer whose size a *_size query returns.
 *  - Every call is ordered on the given stream (a cudaStream_t; NULL = the
 *    legacy default stream) and returns as soon as its work is enqueued.
 *    Nothing synchronises except dt_read_stats (documented there).
 *  - FP32 throughout.  Arrays are row-major and tightly packed:
 *    V float[nv][3], F int32[nf][3] (counter-clockwise seen from outside,
 *    i.e. (v1 - v0) x (v2 - v0) points out of the object), environment
 *    float[env_h][env_w][3] equirectangular with +y up (row 0 = +y pole,
 *    column 0 starts at azimuth 0 = +x, azimuth grows toward +z), images
 *    float[n_views][height][width][3] with row 0 at the top.
 *  - Return value: DT_OK, or an error code with a message in dt_last_error()
 *    (thread-local).  Argument errors are detected on the host before any
 *    work is enqueued.  The contents of device arrays are not inspected on
 *    the host: every entry of F must lie in [0, nv) and V must be finite
 *    (the kernels index V, N and the gradients with F unchecked, so an
 *    out-of-range entry is undefined behaviour).  Errors that only the GPU can see (a full segment
 *    arena, a traversal stack overflow) are recorded in the workspace's
 *    device status word and reported by dt_read_stats; the affected work is
 *    dropped, never written out of bounds.
 */
#ifndef DIFFTRANS_H_
#define DIFFTRANS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int dt_status;
#define DT_OK 0
#define DT_ERR_INVALID_ARG 1
#define DT_ERR_CUDA 2
#define DT_ERR_QUEUE_OVERFLOW 3 /* the segment arena was too small */
#define DT_ERR_STACK_OVERFLOW 4 /* BVH deeper than the traversal stack */
#define DT_ERR_NOT_IMPLEMENTED 5

typedef void* dt_stream; /* cudaStream_t */

/* Message of the last failed call on this thread ("" if none). */
const char* dt_last_error(void);
/* Library version string, "difftrans-gb300 <major>.<minor> (sm_103a)"; the
 * minor number changes with every change of a struct's layout (0.2: dt_medium
 * gained the hash-texture fields). */
const char* dt_version(void);

/* ------------------------------------------------------------------------
 * Vertex normals, Sec. 3.4 Eq. 13: N_v = (1/3) * sum over the faces f that
 * contain v of the unit face normal (v_f1 - v_f0) x (v_f2 - v_f0) / |...|.
 * d_V float[nv][3], d_F int32[nf][3] (every index in [0, nv)), d_N
 * float[nv][3] is overwritten.  The sums are accumulated in 64-bit fixed
 * point (2^-40) in d_scratch (>= dt_vertex_normals_scratch_size bytes,
 * 8-byte aligned, contents undefined afterwards), so the result is the same
 * bits on every run.  A face of zero area has no unit normal and adds
 * nothing to its vertices' normals.
 * ------------------------------------------------------------------------ */
dt_status dt_vertex_normals_scratch_size(int32_t nv, size_t* bytes);
dt_status dt_vertex_normals(const float* d_V, int32_t nv, const int32_t* d_F, int32_t nf, float* d_N,
                            void* d_scratch, dt_stream stream);

/* dt_vertex_normals for callers that cannot allocate device memory: a
 * plugin that only receives device pointers from a host application owning
 * all device memory, or a serving loop that must not allocate after start-up
 * (cudaMalloc/cudaFree can synchronise the device and fragment a pool).  The
 * paper has no counterpart; it computes the same Eq. 13 normals, bit for bit,
 * as dt_vertex_normals, but takes no scratch buffer: it uses one fixed array
 * of 24 MiB of device memory inside the library (2^20 vertices x 3 x 8
 * bytes), which every GPU that loads the library holds until the process
 * exits.  It allocates nothing.
 *  - nv > 1048576 (2^20) is rejected with DT_ERR_INVALID_ARG and a message;
 *    use dt_vertex_normals then.
 *  - The first call in each CUDA context (normally one per device: its
 *    primary context) looks up the array's device address, with that device
 *    current, and keeps it for that context; make that first call before any
 *    stream capture.  A context made anew (after cudaDeviceReset) gets its
 *    own lookup on its first call.
 *  - Every call on a device shares the one array and it keeps the last
 *    call's contents (each call clears the part it uses first).  Calls whose
 *    work overlaps on the GPU -- on different streams, or from different
 *    host threads -- race on it: order them on one stream. */
dt_status dt_vertex_normals_noalloc(const float* d_V, int32_t nv, const int32_t* d_F, int32_t nf, float* d_N,
                                    dt_stream stream);

/* Backward of dt_vertex_normals: d_dV[nv][3] += (dN/dV)^T d_dN, for a
 * gradient d_dN float[nv][3] with respect to the normals.  d_dV is
 * accumulated into, not overwritten. */
dt_status dt_vertex_normals_backward(const float* d_V, int32_t nv, const int32_t* d_F, int32_t nf,
                                     const float* d_dN, float* d_dV, dt_stream stream);

/* ------------------------------------------------------------------------
 * LBVH over the triangles (the paper traces with OptiX, Sec. 3.4; this
 * acceleration structure is the library's own): 30-bit Morton codes of the
 * triangle centroids, a stable radix sort, the Karras (2012) binary
 * hierarchy with one triangle per leaf, then bottom-up bounds.
 *
 * dt_bvh_size: bytes of the BVH buffer and of the build scratch for nf
 *   triangles (nf >= 1).
 * dt_build_bvh: builds into d_bvh (>= bvh_bytes, 256-byte aligned) using
 *   d_scratch (>= scratch_bytes, 256-byte aligned, contents undefined
 *   afterwards).  The BVH keeps no pointer to V or F.
 * dt_refit_bvh: recomputes the bounds and the stored triangle data of an
 *   existing BVH for moved vertices (same F, same nf), keeping the
 *   hierarchy; d_scratch as for the build.
 * ------------------------------------------------------------------------ */
dt_status dt_bvh_size(int32_t nf, size_t* bvh_bytes, size_t* scratch_bytes);
dt_status dt_build_bvh(const float* d_V, int32_t nv, const int32_t* d_F, int32_t nf, void* d_bvh,
                       void* d_scratch, dt_stream stream);
dt_status dt_refit_bvh(const float* d_V, int32_t nv, const int32_t* d_F, int32_t nf, void* d_bvh,
                       void* d_scratch, dt_stream stream);

/* ------------------------------------------------------------------------
 * Scene, views and parameters of a render.
 * ------------------------------------------------------------------------ */
/* Spatially varying absorption (Eq. 11 with mu_t(x) = sigma + G(x)).  On an
 * interior segment (where sigma applies) of length t the optical depth
 * sigma t gains the sum of G over steps of length `step` from the segment's
 * start: m = floor(t / step) full steps (at most 8192) and a last one of
 * length t - m step, each sampled at its midpoint and weighted by its
 * length.  Every lattice below spans the box [lo, hi] and is read with
 * trilinear interpolation at positions clamped to the box.
 *
 * levels == 0: G is a dense grid of per-channel rates at the nodes of an
 * nx x ny x nz lattice (node (i, j, k) at lo + (i, j, k) (hi - lo) / (n - 1)).
 *  d_mu: float[nz][ny][nx][4], 16-byte aligned (the 4th float is unused);
 *  nx, ny, nz >= 2.
 *
 * levels = L in 1..DT_MAX_HASH_LEVELS: G is a multi-resolution hash texture
 * (Sec. 3.3's differentiable 3D texture after Instant-NGP, Mueller et al.
 * 2022): level l is a lattice of res[l] nodes per axis whose values live in
 * the table slice [l T, (l + 1) T), T = 2^log2_table; its corner (i, j, k)
 * is entry (k res + j) res + i when res^3 <= T and otherwise entry
 * (i XOR 2654435761 j XOR 805459861 k) mod T (32-bit unsigned products).
 * G is the sum over the levels of their trilinear interpolations.
 *  d_mu: float[L][T][4], 16-byte aligned (the 4th float is unused);
 *  4 <= log2_table <= 24; 2 <= res[l] <= 2^20; nx, ny, nz ignored.
 *
 *  d_grad_mu: where dt_render_backward writes dLoss/d(node values or table
 *    entries), the layout of d_mu (overwritten; NULL: not computed).  Hash
 *    corners that share an entry add their contributions.
 * hi > lo on every axis; step > 0. */
#define DT_MAX_HASH_LEVELS 16
typedef struct dt_medium {
  const float* d_mu;
  float* d_grad_mu;
  int32_t nx, ny, nz;
  float lo[3], hi[3];
  float step;
  int32_t levels;     /* 0: dense grid; L: hash texture with L levels */
  int32_t log2_table; /* hash texture: log2 of the entries per level */
  int32_t res[DT_MAX_HASH_LEVELS]; /* hash texture: nodes per axis of each level */
} dt_medium;

typedef struct dt_scene {
  const float* d_V;     /* float[nv][3] vertex positions */
  const int32_t* d_F;   /* int32[nf][3] */
  int32_t nv, nf;
  const void* d_bvh;    /* built (or refitted) for exactly these V and F */
  const float* d_N;     /* float[nv][3] vertex normals of V (dt_vertex_normals) */
  const float* d_ior;   /* float[1]: index of refraction of the object (outside = 1) */
  const float* d_sigma; /* float[3]: absorption rate per channel inside the object */
  const float* d_env;   /* float[env_h][env_w][3] environment */
  int32_t env_w, env_h;
  const dt_medium* medium; /* NULL: the constant sigma only */
  float* d_grad_env;       /* backward: dLoss/d(environment texels), float[env_h][env_w][3], overwritten;
                              NULL: not computed (the forward ignores it) */
} dt_scene;

/* n_views pinhole cameras sharing one image size.  d_cams float[n_views][10]
 * = eye xyz, look-at point xyz, up xyz, vertical field of view in degrees.
 * The ray of image point (sx, sy) (pixel px covers sx in [px, px+1)) has
 * origin eye and direction normalize(f + a r + b u) with f = normalize(at -
 * eye), r = normalize(f x up) (f x (0,0,1) if f x up = 0), u = r x f,
 * a = (2 sx / width - 1) tan(fov/2) width/height, b = (1 - 2 sy / height)
 * tan(fov/2). */
typedef struct dt_views {
  const float* d_cams;
  int32_t n_views, width, height;
} dt_views;

/* Parameters.
 *  max_depth: D, the number of surface interactions a path may have
 *    (0 <= D <= 30).  Segments of depth k <= D are intersected; a hit at
 *    depth D contributes nothing (Sec. 3.4 step 1; App. A.3.4 uses 4 in
 *    training and 8 at inference).
 *  spp: samples per pixel (>= 1); pixel = mean over its samples.
 *  jitter: 0 = every sample at the pixel centre; 1 = sample s of pixel p in
 *    view v at p + (hx, hy), hx, hy = the top 24 bits of pcg(h),
 *    pcg(h ^ 0x9E3779B9) times 2^-24, h = pcg(pcg(pcg(pcg(seed_lo ^
 *    pcg(seed_hi)) ^ v) ^ p) ^ s), pcg = the PCG hash of Jarzynski and Olano
 *    (JCGT 2020).
 *  t_min: hits need t > t_min (the triangle a ray leaves from is skipped
 *    as well).  1e-5 for meshes scaled to the unit sphere.
 *  tape_mode: 0 keeps every segment's hit record for the backward; 1 is
 *    per-bounce checkpointing: only the ray queues are kept, the hit
 *    records of the forward live in a ring of two levels of level_capacity
 *    segments each, and the backward recovers the hit of every segment
 *    that spawned children from the source triangle those children carry,
 *    intersecting that one triangle again with the traversal's arithmetic
 *    (16 bytes per segment less, one triangle test per spawning segment
 *    more).  A level larger than level_capacity is dropped past that size
 *    and reported as DT_ERR_QUEUE_OVERFLOW with dt_stats.level_needed.
 *  level_capacity: segments per ring level (tape_mode 1 only; else 0).
 *  tape_mode 2 keeps the full tape of tape_mode 0 and, for every segment that
 *    runs inside the object of a scene with an absorption grid or hash
 *    texture (Eq. 11 with a spatially varying rate), the medium's optical
 *    depth S over the segment, dS/dt and the 3x3 derivatives of S with
 *    respect to the segment's origin and direction (24 floats, 96 bytes per
 *    segment of the arena).  A medium pass of its own computes them between
 *    the traversal and the shading of each level, reading the medium once;
 *    the shading takes S from there and the backward needs no medium value
 *    (only the scatter of dJ/dG into the grid or table marches the segment).
 *    Images and gradients are those of tape_mode 0 up to rounding order.
 *  The workspace must be sized for the same tape_mode and level_capacity
 *  (dt_render_workspace_size_ex) and the backward must be given the same
 *  params as the forward; all entries of a batch share them. */
typedef struct dt_params {
  int32_t max_depth;
  int32_t spp;
  int32_t jitter;
  int32_t tape_mode;
  uint64_t seed;
  float t_min;
  int32_t level_capacity;
} dt_params;

/* ------------------------------------------------------------------------
 * Forward render (Sec. 3.4 steps 1-5), wavefront by depth: camera rays;
 * then for k = 0..D a closest-hit pass over the level-k segments and a
 * shading pass that accumulates escaped rays into the image and appends the
 * reflected and refracted children to level k+1.  Every segment of every
 * level is kept in the workspace (the "tape") for dt_render_backward
 * (tape_mode 1: the ray queues of every level, the hits of the last two).
 *
 * dt_render_workspace_size: bytes for a workspace holding seg_capacity
 *   segments (all levels together; seg_capacity <= 2^31 - 1).  A segment is
 *   one closest-hit query; a pixel sample with a convex object needs at most
 *   2D + 1, any object at most 2^(D+1) - 1.
 * dt_render: d_out float[n_views][height][width][3] is overwritten with the
 *   image.  d_ws (256-byte aligned) of ws_bytes holds the tape afterwards and
 *   must stay untouched until dt_render_backward has run.  When the arena is
 *   too small the excess segments are dropped and the status word records
 *   DT_ERR_QUEUE_OVERFLOW with a lower bound on the capacity needed.
 * ------------------------------------------------------------------------ */
dt_status dt_render_workspace_size(int64_t seg_capacity, size_t* ws_bytes);
/* The same for a tape_mode (see dt_params): tape_mode 1 needs
 * 1 <= level_capacity <= seg_capacity; tape_mode 2 adds 96 bytes per
 * segment (level_capacity ignored). */
dt_status dt_render_workspace_size_ex(int64_t seg_capacity, int32_t tape_mode, int64_t level_capacity,
                                      size_t* ws_bytes);
dt_status dt_render(const dt_scene* scene, const dt_views* views, const dt_params* params, float* d_out,
                    void* d_ws, size_t ws_bytes, dt_stream stream);

/* Statistics of the last dt_render into d_ws (ws_bytes as passed to it).
 * Copies them to host memory, which waits for the stream to reach this point
 * (the one synchronising call).  status is DT_OK or the first device-side
 * error; after DT_ERR_QUEUE_OVERFLOW, seg_needed is a lower bound on the
 * capacity to retry with. */
typedef struct dt_stats {
  int32_t status;
  int32_t n_levels;            /* depth levels that held segments */
  int64_t segments;            /* closest-hit queries traced */
  int64_t seg_needed;          /* lower bound on seg_capacity (overflow) */
  int64_t level_count[32];     /* segments per depth */
  int64_t level_start[32];     /* arena offset of each depth */
  int64_t hits, misses, discarded, backfacing, tir;
  int64_t nodes_visited;       /* BVH nodes whose child boxes were tested */
  int64_t tris_tested;         /* ray/triangle tests */
  int64_t max_level;           /* largest level_count */
  int64_t level_needed;        /* largest level as generated (for tape_mode 1 level_capacity) */
  int64_t medium_samples;      /* absorption-grid samples of the forward (dt_medium) */
} dt_stats;
dt_status dt_read_stats(const void* d_ws, size_t ws_bytes, dt_stats* out, dt_stream stream);

/* ------------------------------------------------------------------------
 * Backward of dt_render: reverse sweep k = D..0 over the tape.  For an image
 * gradient d_grad_out float[n_views][height][width][3] (= dLoss/dImage) it
 * returns the gradient at fixed discrete events (hit triangles,
 * inside/outside, total internal reflection) with respect to the vertex
 * positions, the IoR and sigma, through every term of Sec. 3.3-3.4: the
 * environment lookup, the Fresnel terms (Eqs. 7-8), reflection and
 * refraction (Eqs. 3-6), the interpolated normal (Eq. 12) and the vertex
 * normals (Eq. 13), the barycentric hit point (Sec. 3.4: intersection points
 * interpolated from vertex positions), and the absorption exp(-sigma t).
 *
 * The scene, views and params must be those of the dt_render that filled
 * d_ws (ws_bytes as passed to it), and that render must have finished with
 * status DT_OK; d_ws is only read, and the vertices must not have changed
 * since the forward.  dt_backward_workspace_size: bytes of the backward scratch
 * d_bws (256-byte aligned) for a render whose largest level held max_level
 * segments (dt_stats.max_level); pass the same max_level to
 * dt_render_backward.  Outputs are overwritten: d_grad_V float[nv][3],
 * d_grad_ior float[1], d_grad_sigma float[3].
 * ------------------------------------------------------------------------ */
dt_status dt_backward_workspace_size(int64_t max_level, int32_t nv, size_t* bytes);
dt_status dt_render_backward(const dt_scene* scene, const dt_views* views, const dt_params* params,
                             const void* d_ws, size_t ws_bytes, const float* d_grad_out, float* d_grad_V,
                             float* d_grad_ior, float* d_grad_sigma, void* d_bws, size_t bws_bytes,
                             int64_t max_level, dt_stream stream);

/* ------------------------------------------------------------------------
 * Batching: many scenes of uneven size in one render.  One call traces the
 * camera rays of every scene; then for each depth one persistent traversal
 * launch and one shading launch cover the segments of all scenes together
 * (each segment carries its scene through its sample index), so the number
 * of launches depends on the largest depth only, not on the number of
 * scenes.  Each entry is a scene as for dt_render with its own views,
 * params and image; dt_render is the one-entry batch.  Sample indices are
 * global across the batch (entry i's samples follow entry i-1's) for
 * dt_dump_segments.  n in [1, 256]; the total of primary rays < 2^32.
 * The backward takes d_grad_out, d_grad_V, d_grad_ior, d_grad_sigma of each
 * entry (outputs overwritten) and a scratch sized by
 * dt_batch_backward_workspace_size.  Entries are host memory read during
 * the call; the library keeps no pointer to them.
 * ------------------------------------------------------------------------ */
typedef struct dt_batch_entry {
  dt_scene scene;
  dt_views views;
  dt_params params;
  float* d_out;              /* forward: float[n_views][height][width][3] */
  const float* d_grad_out;   /* backward: dLoss/dImage, same shape */
  float* d_grad_V;           /* backward outputs */
  float* d_grad_ior;
  float* d_grad_sigma;
} dt_batch_entry;
dt_status dt_render_batch(const dt_batch_entry* entries, int32_t n, void* d_ws, size_t ws_bytes, dt_stream stream);
dt_status dt_batch_backward_workspace_size(const dt_batch_entry* entries, int32_t n, int64_t max_level,
                                           size_t* bytes);
dt_status dt_render_batch_backward(const dt_batch_entry* entries, int32_t n, const void* d_ws, size_t ws_bytes,
                                   void* d_bws, size_t bws_bytes, int64_t max_level, dt_stream stream);

/* ------------------------------------------------------------------------
 * Debug / parity: every segment of the tape in arena order (level by
 * level).  d_seg_i int32[cap][4] = (sample index, heap node id, hit triangle
 * or -1, flags); d_seg_f float[cap][15] = (t, b1, b2, origin xyz, direction
 * xyz, throughput W rgb, contribution W * E(d) rgb of a segment that escaped
 * -- Sec. 3.4 step 3 before the 1/spp of the pixel average -- and 0 for a
 * hit); available after a render with tape_mode 0 only (after tape_mode 1
 * or 2 nothing is written).  Sample index = (view*height*width + py*width + px)*spp + s; the
 * heap node id of a camera ray is 1 and the children of node m are 2m
 * (reflected) and 2m+1 (refracted).  Flag bits: 4 inside (hit from inside),
 * 8 total internal reflection, 16 backfacing shading normal, 128 hit at
 * depth D, 512 miss.  Writes min(cap, segments) records.
 * ------------------------------------------------------------------------ */
dt_status dt_dump_segments(const void* d_ws, size_t ws_bytes, int32_t* d_seg_i, float* d_seg_f, int64_t cap,
                           dt_stream stream);

/* Closest hit (Sec. 3.4 step 2) of n arbitrary rays through a BVH built for
 * nf triangles (tooling and tests): d_o, d_d float[n][3]; d_src int32[n]
 * (triangle to skip, -1 for none; may be NULL); hits need t > t_min, ties
 * in t go to the smaller triangle id.  Outputs d_tri int32[n] (-1 = miss,
 * -2 = traversal stack overflow) and d_tbb float[n][3] = (t, b1, b2), the
 * hit point being (1 - b1 - b2) v0 + b1 v1 + b2 v2. */
dt_status dt_closest_hit(const void* d_bvh, int32_t nf, const float* d_o, const float* d_d, const int32_t* d_src,
                         int32_t n, float t_min, int32_t* d_tri, float* d_tbb, dt_stream stream);

/* ------------------------------------------------------------------------
 * Image loss seed for the backward pass.  The paper supervises the rendered
 * colours with an L2 loss (Sec. 3.4 "Optimization"); this is its plain
 * mean-squared form over n values: loss = scale * sum (img - target)^2 and
 * d_grad = 2 scale (img - target), with scale = 1/n for the mean.
 * d_img, d_target, d_grad float[n]; d_loss float[1] is overwritten.
 * ------------------------------------------------------------------------ */
dt_status dt_l2_loss_grad(const float* d_img, const float* d_target, int64_t n, float scale, float* d_grad,
                          float* d_loss, dt_stream stream);

/* The tracer stage's own losses (Sec. 3.4 "Optimization") fused into the
 * backward seed, over n_pix RGB pixels c_hat (rendered) and c (true):
 *   L_color = (1/n_pix) sum_i ||(c_hat_i - c_i) * c_i||^2, the product
 *             channel-wise (Eq. 14);
 *   L_tone  = (1/n_pix) sum_i [(1 - cos(c_hat_i, c_i))^2 - var(c_i)]
 *             (Eq. 15, per pixel: cos of the RGB vectors, 0 when either is
 *             zero; var the population variance of the three true channels).
 * d_img, d_target, d_grad float[n_pix][3]; d_grad = d(total)/d(c_hat) is
 * overwritten; d_loss float[3] = (lambda_color L_color + lambda_tone L_tone,
 * L_color, L_tone) is overwritten.  n_pix = 0 gives zeros (the image
 * pointers may then be NULL). */
dt_status dt_paper_loss_grad(const float* d_img, const float* d_target, int64_t n_pix, float lambda_color,
                             float lambda_tone, float* d_grad, float* d_loss, dt_stream stream);

/* ------------------------------------------------------------------------
 * The step after the gradient (App. A): the paper optimises the mesh with
 * AdamUniform (the optimiser of Nicolet et al. 2021, "Large Steps in
 * Inverse Rendering of Geometry", learning rate 1e-3) and regularises it
 * with the edge term L_edge.
 *
 * Topology: the distinct neighbours of every vertex of a triangle mesh in
 * CSR form, built on the device.  dt_topology_size gives the bytes of the
 * caller buffer (256-byte aligned) for nv vertices and nf triangles;
 * dt_build_topology fills it (indices outside [0, nv) and self-pairs are
 * ignored); dt_topology_info copies the number of distinct edges and the
 * largest neighbour count to the host (synchronising) and, when row/col are
 * given, the device pointers of the CSR arrays (int32 row[nv + 1], col[2 E]).
 *
 * M = I + lambda L with L = D - A the graph Laplacian of those edges
 * (uniform weights).  dt_smooth_solve solves M x = b for b, x float[nv][3]
 * (x holds the start on entry) by conjugate gradients with the diagonal as
 * preconditioner, `iters` iterations, all scalars on the device; scratch
 * of dt_smooth_scratch_size bytes.
 *
 * dt_large_steps_update: one mesh update.  u = M V; g_u = M^-1 dJ/dV (the
 * matrix is symmetric); AdamUniform on u: m = beta1 m + (1 - beta1) g_u,
 * v = beta2 v + (1 - beta2) max_i g_u,i^2 (one second moment for all
 * coordinates), u -= lr (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) +
 * eps); then V = M^-1 u (started from the old V).  d_V float[nv][3] is
 * updated in place; d_state (state_bytes, zeroed by the caller for a fresh
 * optimiser) carries m, v and t between calls; d_scratch of scratch_bytes.
 *
 * dt_edge_loss_grad: L_edge = (1/|E|) sum over distinct edges {i, j} of
 * (1 - n_i . n_j)^2, n the unit vertex normals of d_N (Eq. 13's normals,
 * dt_vertex_normals); d_loss float[1] and d_grad_N = dL_edge/dN float[nv][3]
 * are overwritten (dt_vertex_normals_backward takes it to the vertices).
 * ------------------------------------------------------------------------ */
dt_status dt_topology_size(int32_t nv, int32_t nf, size_t* bytes);
dt_status dt_build_topology(const int32_t* d_F, int32_t nf, int32_t nv, void* d_topo, size_t topo_bytes,
                            dt_stream stream);
dt_status dt_topology_info(const void* d_topo, int32_t nv, int32_t nf, int64_t* n_edges, int32_t* max_degree,
                           const int32_t** d_row, const int32_t** d_col, dt_stream stream);
dt_status dt_smooth_scratch_size(int32_t nv, int32_t iters, size_t* bytes);
dt_status dt_smooth_solve(const void* d_topo, int32_t nv, int32_t nf, float lambda, const float* d_b, float* d_x,
                          int32_t iters, void* d_scratch, size_t scratch_bytes, dt_stream stream);
dt_status dt_large_steps_sizes(int32_t nv, int32_t iters, size_t* state_bytes, size_t* scratch_bytes);
dt_status dt_large_steps_update(const void* d_topo, int32_t nv, int32_t nf, float lambda, float lr, float beta1,
                                float beta2, float eps, int32_t iters, float* d_V, const float* d_grad_V,
                                void* d_state, void* d_scratch, size_t scratch_bytes, dt_stream stream);
dt_status dt_edge_loss_grad(const void* d_topo, int32_t nv, int32_t nf, const float* d_N, float* d_grad_N,
                            float* d_loss, dt_stream stream);

/* ------------------------------------------------------------------------
 * Launch and scheduling knobs of the kernels (process-wide; a call takes
 * the values current when it is made).  The traversal is persistent: each
 * lane carries one ray, a warp runs trace_steps node visits per round and
 * refills its idle lanes from the level's queue once trace_refill of them
 * are idle; trace_blocks_per_sm CTAs of 256 threads run per SM.
 * shade_blocks_per_sm sizes the grid of the shading and adjoint kernels.
 * bvh_width selects the node format the traversal reads: 2 (binary nodes,
 * 64 B) or 4 (4-wide nodes, 128 B: the binary nodes at even depth with
 * their grandchildren as children); both are kept current by build/refit.
 * bvh_builder selects the topology dt_build_bvh builds: 0 = LBVH (Morton
 * codes, radix sort, Karras 2012 hierarchy), 1 = top-down binned surface
 * area heuristic (32 centroid bins per axis, 16 for ranges of at most 128
 * triangles; fewer node visits per ray, slower to build); dt_refit_bvh
 * keeps whichever topology was built.
 * trace_order b (12..22) traces every level after the camera rays bucket
 * by bucket: the bucket is the top b bits of a 24-bit key (direction octant,
 * then the Morton code of the ray origin on a 128^3 grid over the scene's
 * bounding box; in a batch the scene index and the top b-8 bits), counted
 * while the level's segments are shaded into existence and turned into an
 * order by one scan (a counting sort in the level's own not-yet-written
 * hit and flag words), so that a warp's rays take similar paths through the
 * BVH.  0 traces the segments in the order they were appended.  Camera
 * rays are laid out in 8x4 pixel blocks.
 * order_min_rays: a render (or batch) with fewer camera rays than this
 * traces every level in append order: its levels are a few thousand
 * segments, where the order's three launches per level cost more than the
 * coherence gains.
 * Defaults {192, 8, 5, 4, 2, 1, 20, 65536}; results do not depend on them
 * (the same closest hit is found).  dt_set_tuning rejects values outside
 * steps 1..256, refill 1..32, trace 1..8, shade 1..16, width 2 or 4,
 * builder 0 or 1, order 0 or 12..22, order_min_rays >= 0.
 * ------------------------------------------------------------------------ */
typedef struct dt_tuning {
  int32_t trace_steps;
  int32_t trace_refill;
  int32_t trace_blocks_per_sm;
  int32_t shade_blocks_per_sm;
  int32_t bvh_width;
  int32_t bvh_builder;
  int32_t trace_order;
  int32_t order_min_rays;
} dt_tuning;
dt_status dt_get_tuning(dt_tuning* out);
dt_status dt_set_tuning(const dt_tuning* in);

/* ------------------------------------------------------------------------
 * Per-kernel timing.  While enabled, every launch of the library's main
 * kernels is bracketed by CUDA events recorded on its launch stream.
 * dt_profile_read waits for those events, returns per kernel name the
 * number of launches and the summed event time in milliseconds (at most
 * cap entries, *n = number of names), and clears the record.
 * ------------------------------------------------------------------------ */
typedef struct dt_kernel_time {
  char name[40];
  int64_t launches;
  double total_ms;
} dt_kernel_time;
dt_status dt_profile_enable(int32_t enable);
dt_status dt_profile_read(dt_kernel_time* out, int32_t cap, int32_t* n);

/* ------------------------------------------------------------------------
 * Measurement utility (no counterpart in the paper): L2 read bandwidth of
 * the current GPU in GB/s, from float4 loads that bypass L1 over d_buf
 * (bytes >= 4096, 16-byte aligned; choose it well below the L2 size) read
 * iters times after one warming pass.  Synchronises the stream.  The value
 * is the on-chip denominator for kernels whose working set stays in L2.
 * ------------------------------------------------------------------------ */
dt_status dt_measure_l2_read_bandwidth(const void* d_buf, size_t bytes, int32_t iters, double* gbps,
                                       dt_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* DIFFTRANS_H_ */

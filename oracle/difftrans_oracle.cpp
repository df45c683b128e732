// FP64 brute-force oracle for the recursive differentiable transparent-mesh
// tracer of DiffTrans (arXiv 2603.00413, Sec. 3.3 "Light Interaction with
// Transparent Objects" and Sec. 3.4 "Differentiable Mesh Ray Tracer").
//
// TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
// definition the CUDA library is checked against.  Only the tests, the smoke
// check and the CPU-baseline leg of the benchmark may load it; the library
// never calls it and shares no code with it.
//
// What it computes, per pixel sample, is the depth-limited binary ray tree of
// Sec. 3.4 ("Recursive Ray Tracing", steps 1-5), evaluated recursively in
// double precision with a closest-hit search over EVERY triangle (no
// acceleration structure).  Everything is templated on the scalar type so the
// same code, instantiated on forward-mode dual numbers, yields the exact
// directional derivative (JVP) of the rendered image with respect to vertex
// positions, IoR and per-channel absorption at fixed discrete events (hit
// triangles, inside/outside, total internal reflection).
//
// Readings of the paper taken here (each one is listed with its reason in the
// design notes of the repository):
//  * eta is n_transmitted / n_incident (Sec. 3.3, the only reading consistent
//    with Eqs. 4-6); the outside medium has IoR 1.
//  * cos(theta_i) = omega_i . n with n the shading normal turned toward the
//    incoming side; sin^2 = 1 - cos^2.
//  * total internal reflection: R = 1, T = 0 and no refracted child.
//  * depth D counts surface interactions: segments of depth k <= D are
//    intersected; a hit at k = D contributes 0; a miss at any depth returns the
//    environment (an interior miss -- a leak -- unattenuated).
//  * vertex normals follow Eq. 13 literally: (1/3) times the sum of unit face
//    normals, not renormalised; the interpolated shading normal is normalised.
//  * inside/outside from the sign of d . (e1 x e2); if the oriented shading
//    normal faces away from the incoming ray (c <= 0) the node contributes 0.
//  * hit point and barycentrics are functions of (o, d, v0, v1, v2) (the full
//    derivative of the intersection, Sec. 3.4 "Differentiable Mesh
//    Intersection").
//  * absorption with a constant per-channel rate: exp(-sigma * t) over an
//    interior segment of length t (Eq. 11 with one exact step).
//  * optional spatially varying absorption (Eq. 11 with mu_t = sigma + G):
//    G is a dense grid of per-channel node values over a box, trilinear,
//    positions clamped to the box; the segment is cut from its start into
//    steps of length h (the last one partial: t - m h, m = floor(t / h), at
//    most 8192 full steps), each contributing G at its midpoint times its
//    length.  It applies where sigma does: on interior segments.
//  * G may instead be a multi-resolution hash texture (the "differentiable
//    3D texture" of Sec. 3.3, after Instant-NGP, Mueller et al. 2022): L
//    lattices over the same box with n_l nodes per axis, each level's values
//    in its own table of T entries, the corner (i, j, k) of level l stored at
//    ((k n_l + j) n_l + i) when n_l^3 <= T and otherwise at Instant-NGP's
//    spatial hash (i * 1 XOR j * 2654435761 XOR k * 805459861, in 32-bit
//    unsigned arithmetic) modulo T; G is the sum over the levels of their
//    trilinear interpolations, each with three features, the rates
//    themselves (no decoder network).
//  * self-intersection: the triangle a ray leaves from is skipped and hits need
//    t > t_min.  Ties on t go to the smaller triangle id.
//  * environment: equirectangular, y up, bilinear, wrap in u, clamp in v.
//  * camera: pinhole look-at, pixel centres (px + 0.5, py + 0.5), row 0 on top;
//    jitter from the PCG hash of Jarzynski & Olano (JCGT 2020).
#include <cmath>
#include <cstdint>
#include <cstring>
#include <algorithm>
#include <vector>

namespace orc {

// ---------------------------------------------------------------------------
// scalars: double, and dual numbers carrying K tangent components
// ---------------------------------------------------------------------------
template <int K>
struct Dual {
  double v;
  double d[K];
  Dual() : v(0.0) { for (int i = 0; i < K; ++i) d[i] = 0.0; }
  Dual(double x) : v(x) { for (int i = 0; i < K; ++i) d[i] = 0.0; }  // NOLINT
};

inline double val(double x) { return x; }
template <int K> inline double val(const Dual<K>& x) { return x.v; }

template <int K> inline Dual<K> operator+(const Dual<K>& a, const Dual<K>& b) {
  Dual<K> r; r.v = a.v + b.v; for (int i = 0; i < K; ++i) r.d[i] = a.d[i] + b.d[i]; return r; }
template <int K> inline Dual<K> operator-(const Dual<K>& a, const Dual<K>& b) {
  Dual<K> r; r.v = a.v - b.v; for (int i = 0; i < K; ++i) r.d[i] = a.d[i] - b.d[i]; return r; }
template <int K> inline Dual<K> operator-(const Dual<K>& a) {
  Dual<K> r; r.v = -a.v; for (int i = 0; i < K; ++i) r.d[i] = -a.d[i]; return r; }
template <int K> inline Dual<K> operator*(const Dual<K>& a, const Dual<K>& b) {
  Dual<K> r; r.v = a.v * b.v; for (int i = 0; i < K; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i]; return r; }
template <int K> inline Dual<K> operator/(const Dual<K>& a, const Dual<K>& b) {
  Dual<K> r; r.v = a.v / b.v;
  for (int i = 0; i < K; ++i) r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) / (b.v * b.v);
  return r; }
template <int K> inline Dual<K> operator+(const Dual<K>& a, double b) { return a + Dual<K>(b); }
template <int K> inline Dual<K> operator+(double a, const Dual<K>& b) { return Dual<K>(a) + b; }
template <int K> inline Dual<K> operator-(const Dual<K>& a, double b) { return a - Dual<K>(b); }
template <int K> inline Dual<K> operator-(double a, const Dual<K>& b) { return Dual<K>(a) - b; }
template <int K> inline Dual<K> operator*(const Dual<K>& a, double b) { return a * Dual<K>(b); }
template <int K> inline Dual<K> operator*(double a, const Dual<K>& b) { return Dual<K>(a) * b; }
template <int K> inline Dual<K> operator/(const Dual<K>& a, double b) { return a / Dual<K>(b); }
template <int K> inline Dual<K> operator/(double a, const Dual<K>& b) { return Dual<K>(a) / b; }

// each elementary function: value, then derivative by the chain rule
template <int K> inline Dual<K> chain(const Dual<K>& a, double f, double df) {
  Dual<K> r; r.v = f; for (int i = 0; i < K; ++i) r.d[i] = df * a.d[i]; return r; }
template <int K> inline Dual<K> sqrt(const Dual<K>& a) { double s = std::sqrt(a.v); return chain(a, s, 0.5 / s); }
template <int K> inline Dual<K> exp(const Dual<K>& a) { double e = std::exp(a.v); return chain(a, e, e); }
template <int K> inline Dual<K> acos(const Dual<K>& a) {
  return chain(a, std::acos(a.v), -1.0 / std::sqrt(1.0 - a.v * a.v)); }
template <int K> inline Dual<K> atan2(const Dual<K>& y, const Dual<K>& x) {
  Dual<K> r; r.v = std::atan2(y.v, x.v);
  double den = x.v * x.v + y.v * y.v;
  for (int i = 0; i < K; ++i) r.d[i] = (x.v * y.d[i] - y.v * x.d[i]) / den;
  return r; }
using std::sqrt; using std::exp; using std::acos; using std::atan2;

// ---------------------------------------------------------------------------
// 3-vectors
// ---------------------------------------------------------------------------
template <class T>
struct V3 {
  T x, y, z;
  V3() : x(0.0), y(0.0), z(0.0) {}
  V3(T a, T b, T c) : x(a), y(b), z(c) {}
};
template <class T> inline V3<T> operator+(const V3<T>& a, const V3<T>& b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <class T> inline V3<T> operator-(const V3<T>& a, const V3<T>& b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class T> inline V3<T> operator-(const V3<T>& a) { return {-a.x, -a.y, -a.z}; }
template <class T, class S> inline V3<T> operator*(const V3<T>& a, const S& s) { return {a.x * s, a.y * s, a.z * s}; }
template <class T, class S> inline V3<T> operator*(const S& s, const V3<T>& a) { return {a.x * s, a.y * s, a.z * s}; }
template <class T> inline T dot(const V3<T>& a, const V3<T>& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class T> inline V3<T> cross(const V3<T>& a, const V3<T>& b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
template <class T> inline T norm(const V3<T>& a) { return sqrt(dot(a, a)); }
template <class T> inline V3<T> normalize(const V3<T>& a) { T n = norm(a); return {a.x / n, a.y / n, a.z / n}; }
template <class T> inline V3<double> val3(const V3<T>& a) { return {val(a.x), val(a.y), val(a.z)}; }
template <class T> inline T mul(const T& a, const T& b) { return a * b; }

using V3d = V3<double>;

// ---------------------------------------------------------------------------
// Eq. 13: vertex normal = (1/3) * sum over incident faces of the unit normal
// (v1 - v0) x (v2 - v0) / |(v1 - v0) x (v2 - v0)|.  A zero-area face has no
// unit normal and adds nothing.
// ---------------------------------------------------------------------------
template <class T>
void vertex_normals(const std::vector<V3<T>>& V, const int* F, int nf, std::vector<V3<T>>& N) {
  N.assign(V.size(), V3<T>());
  for (int f = 0; f < nf; ++f) {
    const int i0 = F[3 * f], i1 = F[3 * f + 1], i2 = F[3 * f + 2];
    V3<T> c = cross(V[i1] - V[i0], V[i2] - V[i0]);
    if (!(val(dot(c, c)) > 0.0)) continue;
    V3<T> u = normalize(c);
    N[i0] = N[i0] + u; N[i1] = N[i1] + u; N[i2] = N[i2] + u;
  }
  for (auto& n : N) n = n * T(1.0 / 3.0);
}

// ---------------------------------------------------------------------------
// Ray/triangle intersection: the Moller-Trumbore (1997) solution of
// o + t d = v0 + b1 (v1 - v0) + b2 (v2 - v0) by Cramer's rule.
// Returns false when the system is singular (ray parallel to the plane).
// ---------------------------------------------------------------------------
template <class T>
bool solve_ray_triangle(const V3<T>& o, const V3<T>& d, const V3<T>& v0, const V3<T>& v1,
                        const V3<T>& v2, T& t, T& b1, T& b2) {
  V3<T> e1 = v1 - v0, e2 = v2 - v0;
  V3<T> p = cross(d, e2);
  T det = dot(e1, p);
  if (val(det) == 0.0) return false;
  T inv = 1.0 / det;
  V3<T> s = o - v0;
  b1 = dot(s, p) * inv;
  V3<T> q = cross(s, e1);
  b2 = dot(d, q) * inv;
  t = dot(e2, q) * inv;
  return true;
}

// segment flag bits (shared meaning with the parity dumps of the library)
enum : int {
  SEG_NEAR_EDGE = 1,     // hit or a closer near-miss within 1e-6 of a triangle edge
  SEG_NEAR_TIE = 2,      // another triangle within 1e-6 relative in t
  SEG_INSIDE = 4,        // the segment runs inside the object (hit from inside)
  SEG_TIR = 8,           // total internal reflection at the hit
  SEG_BACKFACING = 16,   // oriented shading normal faces away (c <= 0): contributes 0
  SEG_NEAR_CRITICAL = 32,// |eta^2 - sin^2| < 1e-6: TIR decision unstable
  SEG_GRAZING = 64,      // |d . n_g| or |c| below 1e-6: classification unstable
  SEG_DISCARDED = 128,   // hit at depth D: contributes 0
  SEG_NEAR_POLE = 256,   // environment lookup within 1e-6 of a pole
  SEG_MISS = 512,        // no hit: environment lookup
  SEG_UNSTABLE = 1024,   // pixel only: the path's events change when the primary ray is tilted by probe_delta
};
const int SEG_DEGENERATE =
    SEG_NEAR_EDGE | SEG_NEAR_TIE | SEG_NEAR_CRITICAL | SEG_GRAZING | SEG_NEAR_POLE | SEG_UNSTABLE;

struct Hit {
  int tri = -1;
  double t = 0.0, b1 = 0.0, b2 = 0.0;
  int flags = 0;
};

// Closest hit over ALL triangles in double precision: smallest t > t_min,
// skipping the triangle the ray starts on; exact ties go to the smaller id.
// Also flags near-degenerate configurations: a hit within 1e-6 (barycentric)
// of an edge, a closer triangle missed by less than that, or a second hit
// within 1e-6 relative in t.
Hit closest_hit(const std::vector<V3d>& V, const int* F, int nf, const V3d& o, const V3d& d,
                int src, double t_min) {
  const double EPS = 1e-6;
  Hit h;
  double best = INFINITY;
  double near_edge_t = INFINITY;  // smallest t of any near-edge candidate
  double second = INFINITY;       // second smallest hit t
  for (int f = 0; f < nf; ++f) {
    if (f == src) continue;
    double t, b1, b2;
    if (!solve_ray_triangle(o, d, V[F[3 * f]], V[F[3 * f + 1]], V[F[3 * f + 2]], t, b1, b2)) continue;
    if (!(t > t_min)) continue;
    double mb = std::min(std::min(b1, b2), 1.0 - b1 - b2);
    if (std::fabs(mb) < EPS) near_edge_t = std::min(near_edge_t, t);
    if (mb < 0.0) continue;
    if (t < best) {
      second = best;
      best = t;
      h.tri = f; h.t = t; h.b1 = b1; h.b2 = b2;
    } else {
      second = std::min(second, t);
    }
  }
  if (near_edge_t < INFINITY && near_edge_t <= best * (1.0 + EPS)) h.flags |= SEG_NEAR_EDGE;
  if (h.tri >= 0 && second <= best * (1.0 + EPS)) h.flags |= SEG_NEAR_TIE;
  return h;
}

// ---------------------------------------------------------------------------
// Sec. 3.3 at one surface point.  d: incoming ray direction (unit); n: unit
// shading normal on the incoming side (omega_i . n > 0 with omega_i = -d);
// eta1, eta2: IoR of the incident and transmitted media.
// Eq. 3 (reflection), Eqs. 4-6 (refraction), the TIR test, Eqs. 7-8
// (unpolarised Fresnel R and T = 1 - R).  Returns true under TIR.
// ---------------------------------------------------------------------------
template <class T>
bool interface_terms(const V3<T>& d, const V3<T>& n, const T& eta1, const T& eta2, V3<T>& wr,
                     V3<T>& wt, T& R, T& Tt, double* kappa_out = nullptr) {
  V3<T> wi = -d;
  T c = dot(wi, n);                       // cos(theta_i)
  T eta = eta2 / eta1;                    // n_transmitted / n_incident
  wr = 2.0 * c * n - wi;                  // Eq. 3
  T kappa = eta * eta - (1.0 - c * c);    // eta^2 - sin^2(theta_i)
  if (kappa_out) *kappa_out = val(kappa);
  if (val(kappa) < 0.0) {                 // total internal reflection
    R = T(1.0); Tt = T(0.0); wt = V3<T>();
    return true;
  }
  T cos_t = sqrt(kappa) / eta;            // cos(theta_t)
  V3<T> w_par = (-1.0 * cos_t) * n;       // Eq. 5: -n (1/eta) sqrt(eta^2 - sin^2)
  V3<T> w_perp = (wi - c * n) * (-1.0 / eta);  // Eq. 6
  wt = w_perp + w_par;                    // Eq. 4
  T rs = (eta1 * c - eta2 * cos_t) / (eta1 * c + eta2 * cos_t);
  T rp = (eta1 * cos_t - eta2 * c) / (eta1 * cos_t + eta2 * c);
  R = 0.5 * (rs * rs + rp * rp);          // Eq. 7
  Tt = 1.0 - R;                           // Eq. 8
  return false;
}

// ---------------------------------------------------------------------------
// equirectangular environment, y up: phi = atan2(dz, dx) in [0, 2pi),
// theta = acos(dy); texel coordinates u = phi/(2pi) W - 1/2, v = theta/pi H - 1/2;
// bilinear, wrapping in u and clamping in v.  env: [H][W][3].
// ---------------------------------------------------------------------------
template <class T>
V3<T> env_lookup(const double* env, int W, int H, const V3<T>& d, int* flags = nullptr,
                 uint64_t* cell = nullptr) {
  const double PI = 3.14159265358979323846;
  T phi = atan2(d.z, d.x);
  if (val(phi) < 0.0) phi = phi + 2.0 * PI;
  double dy = val(d.y);
  T cy = d.y;
  if (dy > 1.0) cy = T(1.0);
  if (dy < -1.0) cy = T(-1.0);
  if (flags && std::fabs(dy) > 1.0 - 1e-6) *flags |= SEG_NEAR_POLE;
  T theta = acos(cy);
  T u = phi / (2.0 * PI) * double(W) - 0.5;
  T v = theta / PI * double(H) - 0.5;
  double fu = std::floor(val(u)), fv = std::floor(val(v));
  T ax = u - fu, ay = v - fv;
  long x0 = (long)fu, y0 = (long)fv;
  long x1 = x0 + 1, y1 = y0 + 1;
  // the bilinear cell is a discrete event: the lookup is only piecewise smooth
  if (cell) *cell = ((uint64_t)(uint32_t)(x0 + 1) << 32) | (uint64_t)(uint32_t)(y0 + 1);
  x0 = ((x0 % W) + W) % W; x1 = ((x1 % W) + W) % W;
  y0 = std::min(std::max(y0, 0L), (long)H - 1); y1 = std::min(std::max(y1, 0L), (long)H - 1);
  auto tex = [&](long yy, long xx) { const double* p = env + 3 * (yy * W + xx); return V3<T>(T(p[0]), T(p[1]), T(p[2])); };
  T w00 = (1.0 - ax) * (1.0 - ay), w10 = ax * (1.0 - ay), w01 = (1.0 - ax) * ay, w11 = ax * ay;
  return tex(y0, x0) * w00 + tex(y0, x1) * w10 + tex(y1, x0) * w01 + tex(y1, x1) * w11;
}

// ---------------------------------------------------------------------------
// camera rays and jitter
// ---------------------------------------------------------------------------
inline uint32_t pcg_hash(uint32_t v) {  // Jarzynski & Olano, JCGT 9(3), 2020
  uint32_t state = v * 747796405u + 2891336453u;
  uint32_t word = ((state >> ((state >> 28u) + 4u)) ^ state) * 277803737u;
  return (word >> 22u) ^ word;
}

// Sub-pixel offset in [0,1)^2 of sample `s` of pixel `p` in view `view`.
// h = pcg(pcg(pcg(pcg(seed_lo ^ pcg(seed_hi)) ^ view) ^ p) ^ s);
// offset = ((pcg(h) >> 8) * 2^-24, (pcg(h ^ 0x9E3779B9) >> 8) * 2^-24).
inline void jitter_offset(uint64_t seed, uint32_t view, uint32_t p, uint32_t s, double& jx, double& jy) {
  uint32_t h = pcg_hash((uint32_t)seed ^ pcg_hash((uint32_t)(seed >> 32)));
  h = pcg_hash(h ^ view);
  h = pcg_hash(h ^ p);
  h = pcg_hash(h ^ s);
  jx = (double)(pcg_hash(h) >> 8) * (1.0 / 16777216.0);
  jy = (double)(pcg_hash(h ^ 0x9E3779B9u) >> 8) * (1.0 / 16777216.0);
}

// cam = [eye(3), at(3), up(3), fov_y_deg]
inline void camera_ray(const double* cam, int width, int height, double sx, double sy, V3d& o, V3d& d) {
  const double PI = 3.14159265358979323846;
  V3d eye(cam[0], cam[1], cam[2]), at(cam[3], cam[4], cam[5]), up(cam[6], cam[7], cam[8]);
  V3d fwd = normalize(at - eye);
  V3d r = cross(fwd, up);
  if (norm(r) < 1e-12) r = cross(fwd, V3d(0.0, 0.0, 1.0));
  r = normalize(r);
  V3d u = cross(r, fwd);
  double th = std::tan(0.5 * cam[9] * PI / 180.0);
  double aspect = double(width) / double(height);
  double px = (2.0 * sx / width - 1.0) * th * aspect;
  double py = (1.0 - 2.0 * sy / height) * th;
  o = eye;
  d = normalize(fwd + r * px + u * py);
}

// ---------------------------------------------------------------------------
// the recursive tracer (Sec. 3.4 steps 1-5)
// ---------------------------------------------------------------------------
// Absorption field (Eq. 11 with a spatially varying rate) over the box
// [lo, hi].  levels == 0: a dense grid, node values mu[((k ny + j) nx + i) 3
// + c] at lo + (i, j, k) (hi - lo) / (n - 1).  levels = L >= 1: a hash
// texture whose level l has res[l] nodes per axis (node (i, j, k) at lo +
// (i, j, k) (hi - lo) / (res[l] - 1)) and the table mu[(l T + e) 3 + c],
// T = 2^log2_table, e the corner's entry (dense or hashed, see the header).
constexpr int kMaxHashLevels = 16;
struct orc_medium {
  const double* mu;
  int n[3];
  double lo[3], hi[3];
  double step;
  int levels;
  int log2_table;
  int res[kMaxHashLevels];
};

constexpr long kMaxMediumSteps = 8192;

template <class T>
struct Scene {
  int nv = 0, nf = 0;
  const int* F = nullptr;
  std::vector<V3<T>> V;    // positions (carrying tangents)
  std::vector<V3d> Vd;     // their values, for the search
  std::vector<V3<T>> N;    // vertex normals, Eq. 13
  T ior;
  T sigma[3];
  const double* env = nullptr;
  int env_w = 0, env_h = 0;
  int max_depth = 0;
  double t_min = 0.0;
  // absorption field (has_medium false: sigma only)
  bool has_medium = false;
  int gn[3] = {0, 0, 0};
  double glo[3] = {0, 0, 0}, ghi[3] = {0, 0, 0}, gstep = 0.0;
  int glevels = 0;                   // 0: dense grid; L: hash texture
  uint32_t gtable = 0;               // hash texture: entries per level
  int gres[kMaxHashLevels] = {0};    // hash texture: nodes per axis per level
  std::vector<T> gmu;  // dense: [nz][ny][nx][3]; hash texture: [L][T][3]
};

// Instant-NGP's spatial hash of an integer lattice point (Mueller et al.
// 2022, Eq. 4, d = 3): XOR of the coordinates times the primes 1,
// 2654435761 and 805459861, wrapping in 32 bits; the caller reduces it
// modulo the table size.
inline uint32_t ingp_hash(uint32_t i, uint32_t j, uint32_t k) {
  return (i * 1u) ^ (j * 2654435761u) ^ (k * 805459861u);
}

template <class T>
void set_medium(const orc_medium& M, Scene<T>& S) {
  S.has_medium = true;
  for (int a = 0; a < 3; ++a) { S.gn[a] = M.n[a]; S.glo[a] = M.lo[a]; S.ghi[a] = M.hi[a]; }
  S.gstep = M.step;
  S.glevels = M.levels;
  size_t nn;
  if (M.levels > 0) {
    S.gtable = 1u << M.log2_table;
    for (int l = 0; l < M.levels; ++l) S.gres[l] = M.res[l];
    nn = (size_t)M.levels * S.gtable * 3;
  } else {
    nn = (size_t)M.n[0] * M.n[1] * M.n[2] * 3;
  }
  S.gmu.resize(nn);
  for (size_t i = 0; i < nn; ++i) S.gmu[i] = T(M.mu[i]);
}

// The cell of one lattice of n[0] x n[1] x n[2] nodes over the box that
// holds x: its lowest corner i0 and the fractions f, each coordinate clamped
// to the box (the clamped coordinate is a constant, so it carries no
// derivative).
template <class T>
void lattice_cell(const Scene<T>& S, const int n[3], const V3<T>& x, int i0[3], T f[3]) {
  const T xs[3] = {x.x, x.y, x.z};
  for (int a = 0; a < 3; ++a) {
    const double span = (double)(n[a] - 1);
    T u = (xs[a] - S.glo[a]) / (S.ghi[a] - S.glo[a]) * span;
    if (val(u) < 0.0) u = T(0.0);
    if (val(u) > span) u = T(span);
    int i = (int)std::floor(val(u));
    if (i > n[a] - 2) i = n[a] - 2;
    i0[a] = i;
    f[a] = u - (double)i;
  }
}

// Trilinear interpolation at x of one lattice.  entry(i, j, k) is the index
// of node (i, j, k)'s three values in S.gmu (divided by 3).
template <class T, class Entry>
V3<T> lattice_eval(const Scene<T>& S, const int n[3], Entry entry, const V3<T>& x) {
  T f[3];
  int i0[3];
  lattice_cell(S, n, x, i0, f);
  V3<T> acc;
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        const T w = (dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) * (dz ? f[2] : 1.0 - f[2]);
        const size_t node = entry(i0[0] + dx, i0[1] + dy, i0[2] + dz);
        acc = acc + V3<T>(S.gmu[3 * node], S.gmu[3 * node + 1], S.gmu[3 * node + 2]) * w;
      }
  return acc;
}

// The same lattice as a linear map: the eight corners' entries and weights.
template <class Entry>
void lattice_corners(const Scene<double>& S, const int n[3], Entry entry, const V3d& x, int64_t* idx, double* w) {
  double f[3];
  int i0[3];
  lattice_cell(S, n, x, i0, f);
  int q = 0;
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx, ++q) {
        w[q] = (dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) * (dz ? f[2] : 1.0 - f[2]);
        idx[q] = (int64_t)entry(i0[0] + dx, i0[1] + dy, i0[2] + dz);
      }
}

// Entry of the dense grid's node (i, j, k), and of a hash-texture level's.
inline size_t dense_entry(const int n[3], int i, int j, int k) { return ((size_t)k * n[1] + j) * n[0] + i; }
inline size_t level_entry(uint32_t tsize, int l, int r, int i, int j, int k) {
  const bool hashed = (double)r * r * r > (double)tsize;
  const size_t e = hashed ? (size_t)(ingp_hash((uint32_t)i, (uint32_t)j, (uint32_t)k) % tsize)
                          : ((size_t)k * r + j) * r + i;
  return (size_t)l * tsize + e;
}

// G(x): the dense grid's trilinear interpolation, or the sum over the hash
// texture's levels of theirs.
template <class T>
V3<T> grid_eval(const Scene<T>& S, const V3<T>& x) {
  if (S.glevels == 0)
    return lattice_eval(S, S.gn, [&](int i, int j, int k) { return dense_entry(S.gn, i, j, k); }, x);
  V3<T> acc;
  for (int l = 0; l < S.glevels; ++l) {
    const int r = S.gres[l];
    const int n[3] = {r, r, r};
    acc = acc + lattice_eval(S, n, [&](int i, int j, int k) { return level_entry(S.gtable, l, r, i, j, k); }, x);
  }
  return acc;
}

// Optical depth of the grid over the segment o + s d, s in [0, t]: the sum
// of Eq. 11 over steps of length h from the segment's start, the last one
// partial, each sampled at its midpoint.
template <class T>
V3<T> medium_depth(const Scene<T>& S, const V3<T>& o, const V3<T>& d, const T& t) {
  V3<T> sum;
  if (!S.has_medium) return sum;
  const double h = S.gstep;
  long m = (long)std::floor(val(t) / h);
  if (m < 0) m = 0;
  if (m > kMaxMediumSteps) m = kMaxMediumSteps;
  for (long i = 0; i < m; ++i) sum = sum + grid_eval(S, o + d * T((i + 0.5) * h)) * T(h);
  const T r = t - (double)m * h;
  sum = sum + grid_eval(S, o + d * ((double)m * h + 0.5 * r)) * r;
  return sum;
}

struct SegRec {
  int32_t ray, node, tri, flags;
  double t, b1, b2;
  double o[3], d[3];
  double w[3];  // the segment's throughput: the product of A R or A T over its ancestors
  double c[3];  // an escaped segment's contribution w * E(d) to its sample's radiance; 0 otherwise
};

struct PixelState {
  int flags_or = 0;
  uint64_t sig = 1469598103934665603ull;  // FNV-1a over the event signature
  uint64_t path_sig = 1469598103934665603ull;  // the same without environment texel cells
  V3d discard;
  std::vector<SegRec>* segs = nullptr;
  int32_t ray = 0;
  int64_t counters[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // segments, hits, misses, discarded, leaks, backfacing, tir, degenerate
};

inline void sig_mix(uint64_t& h, uint64_t x) {
  for (int i = 0; i < 8; ++i) { h ^= (x >> (8 * i)) & 0xffu; h *= 1099511628211ull; }
}

template <class T>
V3<T> radiance(const Scene<T>& S, const V3<T>& o, const V3<T>& d, int k, uint32_t node, int src,
               bool in_medium, const V3d& W, PixelState& P) {
  Hit h = closest_hit(S.Vd, S.F, S.nf, val3(o), val3(d), src, S.t_min);
  SegRec rec{P.ray, (int32_t)node, h.tri, h.flags, h.t, h.b1, h.b2,
             {val(o.x), val(o.y), val(o.z)}, {val(d.x), val(d.y), val(d.z)}, {W.x, W.y, W.z}, {0.0, 0.0, 0.0}};
  P.counters[0]++;
  V3<T> L;
  if (h.tri < 0) {  // step 3: no intersection -> environment
    rec.flags |= SEG_MISS;
    uint64_t cell = 0;
    L = env_lookup(S.env, S.env_w, S.env_h, d, &rec.flags, &cell);
    const V3d Lv = val3(L);
    rec.c[0] = W.x * Lv.x; rec.c[1] = W.y * Lv.y; rec.c[2] = W.z * Lv.z;
    sig_mix(P.sig, cell);
    P.counters[2]++;
    // an interior miss (a leak through a crack) returns the environment
    // unattenuated, following step 3 literally; it is counted.
    if (in_medium) P.counters[4]++;
  } else {
    P.counters[1]++;
    const int* f = S.F + 3 * h.tri;
    const V3<T>& v0 = S.V[f[0]]; const V3<T>& v1 = S.V[f[1]]; const V3<T>& v2 = S.V[f[2]];
    V3d ng_d = cross(S.Vd[f[1]] - S.Vd[f[0]], S.Vd[f[2]] - S.Vd[f[0]]);
    double dn = dot(val3(d), ng_d);
    const bool entering = dn < 0.0;                 // step 2: from outside or inside
    if (!entering) rec.flags |= SEG_INSIDE;
    if (std::fabs(dn) < 1e-6 * norm(ng_d) * norm(val3(d))) rec.flags |= SEG_GRAZING;
    if (k >= S.max_depth) {                         // step 1: depth reached
      rec.flags |= SEG_DISCARDED;
      P.discard = P.discard + W;
      P.counters[3]++;
    } else {
      T t, b1, b2;                                  // differentiable intersection
      solve_ray_triangle(o, d, v0, v1, v2, t, b1, b2);
      T b0 = 1.0 - b1 - b2;
      V3<T> x = o + d * t;                          // hit point (== sum b_i v_i)
      V3<T> n = normalize(S.N[f[0]] * b0 + S.N[f[1]] * b1 + S.N[f[2]] * b2);  // Eq. 12
      V3<T> ns = entering ? n : -n;
      T c = dot(-d, ns);
      if (std::fabs(val(c)) < 1e-6) rec.flags |= SEG_GRAZING;
      if (val(c) <= 0.0) {
        rec.flags |= SEG_BACKFACING;
        P.discard = P.discard + W;
        P.counters[5]++;
      } else {
        T eta1 = entering ? T(1.0) : S.ior;
        T eta2 = entering ? S.ior : T(1.0);
        V3<T> wr, wt; T R, Tt; double kappa = 0.0;
        bool tir = interface_terms(d, ns, eta1, eta2, wr, wt, R, Tt, &kappa);
        if (std::fabs(kappa) < 1e-6) rec.flags |= SEG_NEAR_CRITICAL;
        if (tir) { rec.flags |= SEG_TIR; P.counters[6]++; }
        // step 5: absorption over this interior segment (Eq. 11: constant sigma,
        // plus the grid's optical depth when there is one)
        V3<T> A(T(1.0), T(1.0), T(1.0));
        if (!entering) {
          if (S.has_medium) {
            const V3<T> G = medium_depth(S, o, d, t);
            A = V3<T>(exp(-1.0 * (S.sigma[0] * t + G.x)), exp(-1.0 * (S.sigma[1] * t + G.y)),
                      exp(-1.0 * (S.sigma[2] * t + G.z)));
          } else {
            A = V3<T>(exp(-1.0 * S.sigma[0] * t), exp(-1.0 * S.sigma[1] * t), exp(-1.0 * S.sigma[2] * t));
          }
        }
        V3d Ad = val3(A);
        const double Rd = val(R), Td = val(Tt);
        V3d Wr(W.x * Ad.x * Rd, W.y * Ad.y * Rd, W.z * Ad.z * Rd);
        V3d Wt(W.x * Ad.x * Td, W.y * Ad.y * Td, W.z * Ad.z * Td);
        // push the record before the children so records come in pre-order
        P.flags_or |= rec.flags;
        sig_mix(P.sig, (uint64_t)node | ((uint64_t)(uint32_t)h.tri << 32));
        sig_mix(P.sig, (uint64_t)(rec.flags & (SEG_INSIDE | SEG_TIR | SEG_BACKFACING | SEG_DISCARDED | SEG_MISS)));
        sig_mix(P.path_sig, (uint64_t)node | ((uint64_t)(uint32_t)h.tri << 32));
        sig_mix(P.path_sig, (uint64_t)(rec.flags & (SEG_INSIDE | SEG_TIR | SEG_BACKFACING | SEG_DISCARDED | SEG_MISS)));
        if (P.segs) P.segs->push_back(rec);
        // step 4: reflected child at node 2m, refracted child at node 2m+1
        // the reflected ray stays on the incoming side, the refracted one crosses
        V3<T> Lr = radiance(S, x, wr, k + 1, 2u * node, h.tri, !entering, Wr, P);
        V3<T> Lt;
        if (!tir) Lt = radiance(S, x, wt, k + 1, 2u * node + 1u, h.tri, entering, Wt, P);
        V3<T> mix = Lr * R + Lt * Tt;
        L = V3<T>(A.x * mix.x, A.y * mix.y, A.z * mix.z);
        if (rec.flags & SEG_DEGENERATE) P.counters[7]++;
        return L;
      }
    }
  }
  P.flags_or |= rec.flags;
  sig_mix(P.sig, (uint64_t)node | ((uint64_t)(uint32_t)h.tri << 32));
  sig_mix(P.sig, (uint64_t)(rec.flags & (SEG_INSIDE | SEG_TIR | SEG_BACKFACING | SEG_DISCARDED | SEG_MISS)));
  sig_mix(P.path_sig, (uint64_t)node | ((uint64_t)(uint32_t)h.tri << 32));
  sig_mix(P.path_sig, (uint64_t)(rec.flags & (SEG_INSIDE | SEG_TIR | SEG_BACKFACING | SEG_DISCARDED | SEG_MISS)));
  if (rec.flags & SEG_DEGENERATE) P.counters[7]++;
  if (P.segs) P.segs->push_back(rec);
  return L;
}

struct Inputs {
  const double* V; int nv; const int* F; int nf;
  double ior; const double* sigma;
  const double* env; int env_w; int env_h;
  const double* cam; int width; int height;
  int max_depth; int spp; int jitter; uint64_t seed; int view; double t_min;
  const orc_medium* medium;
};

template <class T>
void setup_scene(const Inputs& in, Scene<T>& S) {
  S.nv = in.nv; S.nf = in.nf; S.F = in.F;
  S.V.resize(in.nv); S.Vd.resize(in.nv);
  for (int i = 0; i < in.nv; ++i) {
    S.V[i] = V3<T>(T(in.V[3 * i]), T(in.V[3 * i + 1]), T(in.V[3 * i + 2]));
    S.Vd[i] = V3d(in.V[3 * i], in.V[3 * i + 1], in.V[3 * i + 2]);
  }
  S.ior = T(in.ior);
  for (int c = 0; c < 3; ++c) S.sigma[c] = T(in.sigma[c]);
  S.env = in.env; S.env_w = in.env_w; S.env_h = in.env_h;
  S.max_depth = in.max_depth; S.t_min = in.t_min;
  if (in.medium && in.medium->mu) set_medium(*in.medium, S);
}

// Render a set of pixels.  Pixel p has `spp` primary rays; ray_od(p, s, o, d)
// gives them.  Pixel value = mean over its samples of the radiance of the
// primary ray (step 5 of the tree definition).
template <class T, class RayFn>
void render_pixels(int npix, int spp, const Scene<T>& S, RayFn ray_od, std::vector<V3<T>>& img,
                   std::vector<PixelState>& ps, bool keep_segs, std::vector<std::vector<SegRec>>& segs) {
  img.assign(npix, V3<T>());
  ps.assign(npix, PixelState());
  if (keep_segs) segs.assign(npix, std::vector<SegRec>());
#pragma omp parallel for schedule(dynamic, 16)
  for (int p = 0; p < npix; ++p) {
    PixelState& P = ps[p];
    if (keep_segs) P.segs = &segs[p];
    V3<T> acc;
    for (int s = 0; s < spp; ++s) {
      V3d o, d;
      ray_od(p, s, o, d);
      P.ray = p * spp + s;
      V3<T> L = radiance(S, V3<T>(T(o.x), T(o.y), T(o.z)), V3<T>(T(d.x), T(d.y), T(d.z)), 0, 1u, -1,
                         false, V3d(1.0, 1.0, 1.0), P);
      acc = acc + L;
    }
    img[p] = acc * T(1.0 / spp);
    P.discard = P.discard * (1.0 / spp);
  }
}

// Stability probe: re-trace every sample's primary ray and four copies of it
// tilted by delta radians (two orthogonal axes, both signs).  A pixel is
// flagged SEG_UNSTABLE when, for any copy, the path signature (hit triangles
// and inside/TIR/backfacing/depth/miss events, not the environment cells)
// differs, or the radiance moves by more than rel_tol relative.  It marks the
// paths that pass so close to an edge, or so near a singular point of the
// optics (the TIR critical angle), that a tracer carrying slightly different
// rounding may take another branch or land far away.
template <class RayFn>
void probe_stability(int npix, int spp, const Scene<double>& S, RayFn ray_od, double delta,
                     std::vector<PixelState>& ps, double rel_tol = 1e-4) {
#pragma omp parallel for schedule(dynamic, 16)
  for (int p = 0; p < npix; ++p) {
    for (int s = 0; s < spp; ++s) {
      V3d o, d;
      ray_od(p, s, o, d);
      V3d a = std::fabs(d.x) < 0.9 ? V3d(1.0, 0.0, 0.0) : V3d(0.0, 1.0, 0.0);
      V3d t1 = normalize(cross(d, a)), t2 = cross(d, t1);
      uint64_t ref = 0;
      V3d L0;
      for (int q = 0; q < 5; ++q) {
        V3d dq = d;
        if (q > 0) {
          const double sg = (q & 1) ? delta : -delta;
          dq = normalize(d + ((q <= 2) ? t1 : t2) * sg);
        }
        PixelState P;
        V3d L = radiance(S, o, dq, 0, 1u, -1, false, V3d(1.0, 1.0, 1.0), P);
        if (q == 0) {
          ref = P.path_sig;
          L0 = L;
          continue;
        }
        const double dx = std::fabs(L.x - L0.x), dy = std::fabs(L.y - L0.y), dz = std::fabs(L.z - L0.z);
        if (P.path_sig != ref || dx > rel_tol * std::fabs(L0.x) + 1e-12 || dy > rel_tol * std::fabs(L0.y) + 1e-12 ||
            dz > rel_tol * std::fabs(L0.z) + 1e-12) {
          ps[p].flags_or |= SEG_UNSTABLE;
          break;
        }
      }
      if (ps[p].flags_or & SEG_UNSTABLE) break;
    }
  }
}

template <class T>
void render_view(const Inputs& in, const Scene<T>& S, std::vector<V3<T>>& img, std::vector<PixelState>& ps,
                 bool keep_segs, std::vector<std::vector<SegRec>>& segs) {
  auto cam_ray = [&](int p, int s, V3d& o, V3d& d) {
    double jx = 0.5, jy = 0.5;
    if (in.jitter) jitter_offset(in.seed, (uint32_t)in.view, (uint32_t)p, (uint32_t)s, jx, jy);
    camera_ray(in.cam, in.width, in.height, (p % in.width) + jx, (p / in.width) + jy, o, d);
  };
  render_pixels(in.width * in.height, in.spp, S, cam_ray, img, ps, keep_segs, segs);
}

}  // namespace orc

using namespace orc;

extern "C" {

int orc_version(void) { return 1; }

// Eq. 13 vertex normals.  V: [nv][3], F: [nf][3], N out: [nv][3].
int orc_vertex_normals(const double* V, int nv, const int* F, int nf, double* N) {
  std::vector<V3d> Vv(nv), Nv;
  for (int i = 0; i < nv; ++i) Vv[i] = V3d(V[3 * i], V[3 * i + 1], V[3 * i + 2]);
  vertex_normals(Vv, F, nf, Nv);
  for (int i = 0; i < nv; ++i) { N[3 * i] = Nv[i].x; N[3 * i + 1] = Nv[i].y; N[3 * i + 2] = Nv[i].z; }
  return 0;
}

// Brute-force closest hit for n rays (o, d: [n][3]; src: [n] triangle to skip
// or -1).  Outputs tri (-1 = miss), t, b1, b2, flags.
int orc_closest_hit(const double* V, int nv, const int* F, int nf, const double* o, const double* d,
                    const int* src, int n, double t_min, int* tri, double* t, double* b1, double* b2,
                    int* flags) {
  std::vector<V3d> Vv(nv);
  for (int i = 0; i < nv; ++i) Vv[i] = V3d(V[3 * i], V[3 * i + 1], V[3 * i + 2]);
#pragma omp parallel for schedule(dynamic, 64)
  for (int r = 0; r < n; ++r) {
    Hit h = closest_hit(Vv, F, nf, V3d(o[3 * r], o[3 * r + 1], o[3 * r + 2]),
                        V3d(d[3 * r], d[3 * r + 1], d[3 * r + 2]), src ? src[r] : -1, t_min);
    tri[r] = h.tri; t[r] = h.t; b1[r] = h.b1; b2[r] = h.b2; flags[r] = h.flags;
  }
  return 0;
}

// Sec. 3.3 at one interface for n configurations: d, n: [n][3], eta1, eta2: [n].
// Outputs wr, wt: [n][3]; R, T: [n]; tir: [n].
int orc_interface(const double* d, const double* nrm, const double* eta1, const double* eta2, int n,
                  double* wr, double* wt, double* R, double* T, int* tir) {
  for (int i = 0; i < n; ++i) {
    V3d dd(d[3 * i], d[3 * i + 1], d[3 * i + 2]), nn(nrm[3 * i], nrm[3 * i + 1], nrm[3 * i + 2]);
    V3d r, t; double RR, TT;
    tir[i] = interface_terms(dd, nn, eta1[i], eta2[i], r, t, RR, TT) ? 1 : 0;
    wr[3 * i] = r.x; wr[3 * i + 1] = r.y; wr[3 * i + 2] = r.z;
    wt[3 * i] = t.x; wt[3 * i + 1] = t.y; wt[3 * i + 2] = t.z;
    R[i] = RR; T[i] = TT;
  }
  return 0;
}

// Environment lookup for n directions d: [n][3] -> rgb [n][3].
int orc_env_lookup(const double* env, int W, int H, const double* d, int n, double* rgb) {
  for (int i = 0; i < n; ++i) {
    V3d c = env_lookup(env, W, H, V3d(d[3 * i], d[3 * i + 1], d[3 * i + 2]));
    rgb[3 * i] = c.x; rgb[3 * i + 1] = c.y; rgb[3 * i + 2] = c.z;
  }
  return 0;
}

// Camera rays of one view: o, d: [H*W*spp][3], ray index = (py*W + px)*spp + s.
int orc_camera_rays(const double* cam, int width, int height, int spp, int jitter, uint64_t seed, int view,
                    double* o, double* d) {
  for (int p = 0; p < width * height; ++p) {
    for (int s = 0; s < spp; ++s) {
      double jx = 0.5, jy = 0.5;
      if (jitter) jitter_offset(seed, (uint32_t)view, (uint32_t)p, (uint32_t)s, jx, jy);
      V3d oo, dd;
      camera_ray(cam, width, height, (p % width) + jx, (p / width) + jy, oo, dd);
      const int r = p * spp + s;
      o[3 * r] = oo.x; o[3 * r + 1] = oo.y; o[3 * r + 2] = oo.z;
      d[3 * r] = dd.x; d[3 * r + 1] = dd.y; d[3 * r + 2] = dd.z;
    }
  }
  return 0;
}

uint32_t orc_pcg_hash(uint32_t v) { return pcg_hash(v); }

// doubles per segment in seg_f: t, b1, b2, origin xyz, direction xyz,
// throughput rgb, escaped contribution rgb
constexpr int kSegF = 15;

static int write_outputs(int npix, const std::vector<V3d>& im, const std::vector<PixelState>& ps,
                         const std::vector<std::vector<SegRec>>& segs, bool keep, double* img, double* discard,
                         int* pix_flags, uint64_t* pix_sig, int32_t* seg_i, double* seg_f, int64_t cap,
                         int64_t* n_seg, int64_t* counters) {
  int64_t total = 0;
  int64_t cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int p = 0; p < npix; ++p) {
    img[3 * p] = im[p].x; img[3 * p + 1] = im[p].y; img[3 * p + 2] = im[p].z;
    if (discard) { discard[3 * p] = ps[p].discard.x; discard[3 * p + 1] = ps[p].discard.y; discard[3 * p + 2] = ps[p].discard.z; }
    if (pix_flags) pix_flags[p] = ps[p].flags_or;
    if (pix_sig) pix_sig[p] = ps[p].sig;
    for (int c = 0; c < 8; ++c) cnt[c] += ps[p].counters[c];
    if (keep) {
      for (const SegRec& r : segs[p]) {
        if (seg_i && total < cap) {
          int32_t* si = seg_i + 4 * total;
          si[0] = r.ray; si[1] = r.node; si[2] = r.tri; si[3] = r.flags;
          if (seg_f) {
            double* sf = seg_f + kSegF * total;
            sf[0] = r.t; sf[1] = r.b1; sf[2] = r.b2;
            for (int c = 0; c < 3; ++c) {
              sf[3 + c] = r.o[c]; sf[6 + c] = r.d[c]; sf[9 + c] = r.w[c]; sf[12 + c] = r.c[c];
            }
          }
        }
        ++total;
      }
    }
  }
  if (n_seg) *n_seg = total;
  if (counters) for (int c = 0; c < 8; ++c) counters[c] = cnt[c];
  return (seg_i && total > cap) ? 1 : 0;
}

// Render one view in FP64.
//  img: [H*W][3] radiance; discard (nullable): [H*W][3] path weight lost to
//  depth termination or to a backfacing shading normal (spp-averaged);
//  pix_flags (nullable): OR of segment flags per pixel; pix_sig (nullable):
//  hash of the event signature per pixel; seg_i (nullable): [cap][4] = (ray,
//  heap node, tri, flags) in pixel order, pre-order within a pixel; seg_f:
//  [cap][15] = (t, b1, b2, origin xyz, direction xyz, throughput rgb, the
//  escaped contribution throughput * E(d) rgb, 0 for a hit); n_seg: number of
//  segments (written even when cap is too small); counters (nullable): [8] =
//  segments, hits, misses, discarded, leaks, backfacing, tir, degenerate.
// Returns 0, or 1 when cap was too small (n_seg tells how many are needed).
int orc_render(const double* V, int nv, const int* F, int nf, double ior, const double* sigma,
               const double* env, int env_w, int env_h, const double* cam, int width, int height,
               int max_depth, int spp, int jitter, uint64_t seed, int view, double t_min, double probe_delta,
               double* img, double* discard, int* pix_flags, uint64_t* pix_sig,
               int32_t* seg_i, double* seg_f, int64_t cap, int64_t* n_seg, int64_t* counters,
               const orc_medium* medium) {
  Inputs in{V, nv, F, nf, ior, sigma, env, env_w, env_h, cam, width, height, max_depth, spp, jitter, seed,
            view, t_min, medium};
  Scene<double> S;
  setup_scene(in, S);
  vertex_normals(S.V, F, nf, S.N);
  std::vector<V3d> im;
  std::vector<PixelState> ps;
  std::vector<std::vector<SegRec>> segs;
  const bool keep = seg_i != nullptr || n_seg != nullptr;
  render_view(in, S, im, ps, keep, segs);
  if (probe_delta > 0.0) {
    auto cam_ray = [&](int p, int s, V3d& o, V3d& d) {
      double jx = 0.5, jy = 0.5;
      if (jitter) jitter_offset(seed, (uint32_t)view, (uint32_t)p, (uint32_t)s, jx, jy);
      camera_ray(cam, width, height, (p % width) + jx, (p / width) + jy, o, d);
    };
    probe_stability(width * height, spp, S, cam_ray, probe_delta, ps);
  }
  return write_outputs(width * height, im, ps, segs, keep, img, discard, pix_flags, pix_sig, seg_i, seg_f,
                       cap, n_seg, counters);
}

// The same tree for n arbitrary primary rays (o, d: [n][3], d unit), one
// sample each; outputs as orc_render with npix = n.
int orc_render_rays(const double* V, int nv, const int* F, int nf, double ior, const double* sigma,
                    const double* env, int env_w, int env_h, const double* o, const double* d, int n,
                    int max_depth, double t_min, double probe_delta, double* img, double* discard, int* pix_flags,
                    uint64_t* pix_sig, int32_t* seg_i, double* seg_f, int64_t cap, int64_t* n_seg,
                    int64_t* counters, const orc_medium* medium) {
  Inputs in{V, nv, F, nf, ior, sigma, env, env_w, env_h, nullptr, n, 1, max_depth, 1, 0, 0, 0, t_min, medium};
  Scene<double> S;
  setup_scene(in, S);
  vertex_normals(S.V, F, nf, S.N);
  std::vector<V3d> im;
  std::vector<PixelState> ps;
  std::vector<std::vector<SegRec>> segs;
  const bool keep = seg_i != nullptr || n_seg != nullptr;
  auto given = [&](int p, int, V3d& oo, V3d& dd) {
    oo = V3d(o[3 * p], o[3 * p + 1], o[3 * p + 2]);
    dd = V3d(d[3 * p], d[3 * p + 1], d[3 * p + 2]);
  };
  render_pixels(n, 1, S, given, im, ps, keep, segs);
  if (probe_delta > 0.0) probe_stability(n, 1, S, given, probe_delta, ps);
  return write_outputs(n, im, ps, segs, keep, img, discard, pix_flags, pix_sig, seg_i, seg_f, cap, n_seg,
                       counters);
}

// One step of the tree from given segments, for parity at every depth:
// segment i starts at o_i in the unit direction d_i, leaves triangle src_i
// (-1: none) and has depth index k_i (its number of earlier surface
// interactions).  Its closest hit, its shading (Sec. 3.4 steps 1-5) and its
// children's first intersections follow the tree definition exactly as in
// orc_render; the recursion stops after the children (a child's own hit is
// then counted as discarded).  Each segment starts with throughput 1.
// seg_i: [n][3][4] = (i, heap node 1 / 2 / 3, tri, flags) for the segment
// and its reflected and refracted child, node 0 where there is none;
// seg_f: [n][3][15] as orc_render's records.
int orc_trace_steps(const double* V, int nv, const int* F, int nf, double ior, const double* sigma,
                    const double* env, int env_w, int env_h, const double* o, const double* d, const int* src,
                    const int* k, int n, int max_depth, double t_min, int32_t* seg_i, double* seg_f,
                    const orc_medium* medium) {
  Inputs in{V, nv, F, nf, ior, sigma, env, env_w, env_h, nullptr, n, 1, max_depth, 1, 0, 0, 0, t_min, medium};
  Scene<double> S;
  setup_scene(in, S);
  vertex_normals(S.V, F, nf, S.N);
  for (int64_t j = 0; j < (int64_t)n * 3 * 4; ++j) seg_i[j] = 0;
  for (int64_t j = 0; j < (int64_t)n * 3 * kSegF; ++j) seg_f[j] = 0.0;
#pragma omp parallel for schedule(dynamic, 16)
  for (int i = 0; i < n; ++i) {
    std::vector<SegRec> recs;
    PixelState P;
    P.segs = &recs;
    P.ray = i;
    // the depth test is the only use of the depth index: a segment below
    // the limit is shaded and its children are intersected at the limit
    const int kk = k[i] < max_depth ? max_depth - 1 : max_depth;
    radiance(S, V3d(o[3 * i], o[3 * i + 1], o[3 * i + 2]), V3d(d[3 * i], d[3 * i + 1], d[3 * i + 2]), kk, 1u,
             src ? src[i] : -1, false, V3d(1.0, 1.0, 1.0), P);
    for (const SegRec& r : recs) {
      if (r.node < 1 || r.node > 3) continue;
      const int64_t slot = (int64_t)i * 3 + (r.node - 1);
      int32_t* si = seg_i + 4 * slot;
      si[0] = i; si[1] = r.node; si[2] = r.tri; si[3] = r.flags;
      double* sf = seg_f + kSegF * slot;
      sf[0] = r.t; sf[1] = r.b1; sf[2] = r.b2;
      for (int c = 0; c < 3; ++c) {
        sf[3 + c] = r.o[c]; sf[6 + c] = r.d[c]; sf[9 + c] = r.w[c]; sf[12 + c] = r.c[c];
      }
    }
  }
  return 0;
}

}  // extern "C"

namespace orc {
// Forward-mode derivative along ntan tangent directions, 32 per pass; each
// pass re-runs the tree with dual numbers.  ray_od gives the primary rays.
template <class RayFn>
void jvp_passes(const Inputs& in, int npix, int spp, RayFn ray_od, int ntan, const double* tV,
                       const double* tior, const double* tsigma, const double* tmu, double* img, double* dimg) {
  constexpr int K = 32;
  const int nv = in.nv;
  for (int base = 0; base < ntan; base += K) {
    const int kk = std::min(K, ntan - base);
    Scene<Dual<K>> S;
    setup_scene(in, S);
    for (int j = 0; j < kk; ++j) {
      const int g = base + j;
      if (tV) for (int i = 0; i < nv; ++i) {
        S.V[i].x.d[j] = tV[((size_t)g * nv + i) * 3 + 0];
        S.V[i].y.d[j] = tV[((size_t)g * nv + i) * 3 + 1];
        S.V[i].z.d[j] = tV[((size_t)g * nv + i) * 3 + 2];
      }
      if (tior) S.ior.d[j] = tior[g];
      if (tsigma) for (int c = 0; c < 3; ++c) S.sigma[c].d[j] = tsigma[3 * g + c];
      if (tmu && S.has_medium) {
        const size_t nn = S.gmu.size();
        for (size_t i = 0; i < nn; ++i) S.gmu[i].d[j] = tmu[(size_t)g * nn + i];
      }
    }
    vertex_normals(S.V, in.F, in.nf, S.N);
    std::vector<V3<Dual<K>>> im;
    std::vector<PixelState> ps;
    std::vector<std::vector<SegRec>> segs;
    render_pixels(npix, spp, S, ray_od, im, ps, false, segs);
    for (int p = 0; p < npix; ++p) {
      if (img && base == 0) { img[3 * p] = im[p].x.v; img[3 * p + 1] = im[p].y.v; img[3 * p + 2] = im[p].z.v; }
      for (int j = 0; j < kk; ++j) {
        double* o = dimg + ((size_t)(base + j) * npix + p) * 3;
        o[0] = im[p].x.d[j]; o[1] = im[p].y.d[j]; o[2] = im[p].z.d[j];
      }
    }
  }
}
}  // namespace orc

extern "C" {

// Forward-mode derivative of one view's image along ntan directions at once.
// tV: [ntan][nv][3], tior: [ntan], tsigma: [ntan][3], tmu: [ntan][grid nodes or table entries][3]
// (each nullable = 0; medium nullable = no absorption grid).
// img: [H*W][3] (the same values as orc_render); dimg: [ntan][H*W][3].
int orc_render_jvp(const double* V, int nv, const int* F, int nf, double ior, const double* sigma,
                   const double* env, int env_w, int env_h, const double* cam, int width, int height,
                   int max_depth, int spp, int jitter, uint64_t seed, int view, double t_min,
                   int ntan, const double* tV, const double* tior, const double* tsigma,
                   double* img, double* dimg, const orc_medium* medium, const double* tmu) {
  Inputs in{V, nv, F, nf, ior, sigma, env, env_w, env_h, cam, width, height, max_depth, spp, jitter, seed,
            view, t_min, medium};
  auto cam_ray = [&](int p, int s, V3d& o, V3d& d) {
    double jx = 0.5, jy = 0.5;
    if (jitter) jitter_offset(seed, (uint32_t)view, (uint32_t)p, (uint32_t)s, jx, jy);
    camera_ray(cam, width, height, (p % width) + jx, (p / width) + jy, o, d);
  };
  jvp_passes(in, width * height, spp, cam_ray, ntan, tV, tior, tsigma, tmu, img, dimg);
  return 0;
}

// The same for n arbitrary primary rays (o, d: [n][3]); img: [n][3];
// dimg: [ntan][n][3].
int orc_render_rays_jvp(const double* V, int nv, const int* F, int nf, double ior, const double* sigma,
                        const double* env, int env_w, int env_h, const double* o, const double* d, int n,
                        int max_depth, double t_min, int ntan, const double* tV, const double* tior,
                        const double* tsigma, double* img, double* dimg, const orc_medium* medium,
                        const double* tmu) {
  Inputs in{V, nv, F, nf, ior, sigma, env, env_w, env_h, nullptr, n, 1, max_depth, 1, 0, 0, 0, t_min, medium};
  auto given = [&](int p, int, V3d& oo, V3d& dd) {
    oo = V3d(o[3 * p], o[3 * p + 1], o[3 * p + 2]);
    dd = V3d(d[3 * p], d[3 * p + 1], d[3 * p + 2]);
  };
  jvp_passes(in, n, 1, given, ntan, tV, tior, tsigma, tmu, img, dimg);
  return 0;
}

// The absorption field at n points x ([n][3]): G(x) into out ([n][3]), the
// value the renderer's sum samples.
int orc_field_eval(const orc_medium* medium, const double* x, int n, double* out) {
  Scene<double> S;
  if (!medium || !medium->mu) return 1;
  set_medium(*medium, S);
  for (int p = 0; p < n; ++p) {
    const V3d G = grid_eval(S, V3d(x[3 * p], x[3 * p + 1], x[3 * p + 2]));
    out[3 * p] = G.x; out[3 * p + 1] = G.y; out[3 * p + 2] = G.z;
  }
  return 0;
}

// G as a linear map of the node values or table entries: for each of n
// points, K = 8 max(1, levels) corners (level by level, x fastest within a
// cell) with their entry (a row of the [entries][3] values) and trilinear
// weight: idx, w [n][K].
int orc_field_corners(const orc_medium* medium, const double* x, int n, int64_t* idx, double* w) {
  Scene<double> S;
  if (!medium || !medium->mu) return 1;
  set_medium(*medium, S);
  const int K = 8 * std::max(1, S.glevels);
  for (int p = 0; p < n; ++p) {
    const V3d xp(x[3 * p], x[3 * p + 1], x[3 * p + 2]);
    int64_t* ip = idx + (size_t)p * K;
    double* wp = w + (size_t)p * K;
    if (S.glevels == 0) {
      lattice_corners(S, S.gn, [&](int i, int j, int k) { return dense_entry(S.gn, i, j, k); }, xp, ip, wp);
      continue;
    }
    for (int l = 0; l < S.glevels; ++l) {
      const int r = S.gres[l];
      const int nn[3] = {r, r, r};
      lattice_corners(S, nn, [&](int i, int j, int k) { return level_entry(S.gtable, l, r, i, j, k); }, xp,
                      ip + 8 * l, wp + 8 * l);
    }
  }
  return 0;
}

// Optical depth of the absorption grid over n segments o + s d, s in [0, t]
// (o, d: [n][3], t: [n]); out: [n][3].  The quadrature of Eq. 11 the
// renderer applies to interior segments.
int orc_medium_depth(const orc_medium* medium, const double* o, const double* d, const double* t, int n,
                     double* out) {
  Scene<double> S;
  if (medium && medium->mu) set_medium(*medium, S);
  for (int r = 0; r < n; ++r) {
    const V3d G = medium_depth(S, V3d(o[3 * r], o[3 * r + 1], o[3 * r + 2]), V3d(d[3 * r], d[3 * r + 1], d[3 * r + 2]),
                               t[r]);
    out[3 * r] = G.x; out[3 * r + 1] = G.y; out[3 * r + 2] = G.z;
  }
  return 0;
}

}  // extern "C"

// lt_oracle.cpp -- FP64 CPU oracle for differentiable light tracing.
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or load this
// file; only the test-suite, the smoke check and the CPU-baseline leg of the benchmark
// use it.  It shares no code with the CUDA implementation: its own scene traversal
// (brute force over all primitives), its own Philox4x32-10, its own tape-based
// reverse-mode automatic differentiation.
//
// What it computes (paper section references are to "Constant-Memory Differentiable
// Light Tracing"):
//   * or_render_lt   the light-traced image: every light path x0..xk splats each
//                    unoccluded non-specular vertex connection L_i at film position u_i
//                    through a tent reconstruction filter (Sec. 3.1, Eq. 1-2, Eq. 20).
//   * or_gradient    method 0: naive reverse-mode AD of <dI, I_s(theta)> for a fixed
//                    adjoint image dI, a tape over the whole path (Sec. 3.2, "naive AD").
//                    method 1: LRB-3-pass restated in its three-pass form, detached only
//                    (Sec. 4.3.1, Eq. 14-17).
//                    method 2: naive AD of the ResLRB per-path estimator
//                    S = (Omega_k / w_R) L_R with the weight held constant (Sec. 4.2, Eq. 9-11).
//                    method 3: ResLRB restated in its replay form, detached only (Eq. 11).
//   * or_render_pt   a camera-side path tracer with next-event estimation, used only to
//                    pin the light tracer's normalisation by reciprocity.
//   * or_render_bidir, or_gradient_bidir  a bidirectional estimator: light-tracer sensor
//                    connections and camera samples with next-event estimation, combined
//                    with the balance heuristic, and naive tape AD of it (detached).
//   * helpers exported for pinning tests: Philox, dielectric sampling, reservoir draw,
//                    the frozen-decision loss (for finite differences), and every sensor
//                    connection's values (or_connections: the training pairs of the
//                    learned reservoir target are built from them).
//   * every method optionally applies Russian roulette with a fixed survival probability
//     (see trace()), the path-termination rule the CUDA path replays identically, and
//     either the tent or a wider truncated-Gaussian reconstruction filter (filter_taps).
//
// Model (the "frozen-decision" function that every method differentiates): every
// discrete choice of a path (which primitive each ray hits, reflect/refract branch,
// connection validity, reservoir winner) is taken at the current parameters and held
// fixed.  Vertices that follow the emitter or a non-specular vertex keep their surface
// coordinates (attached samples, Sec. 3.3); their segment weight carries the ratio
// G(theta) A(theta) / [G A](theta0) of the geometry term and triangle area, so that the
// estimator stays a valid estimator as the surface moves.  Vertices that follow a
// specular vertex are re-intersected with the same primitive's plane along the reflected
// or refracted ray (they slide).  Dielectric branch weights are F/F0 and (1-F)/(1-F0).
// Detached mode treats the geometry as constant.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <unordered_map>
#include <vector>

extern "C" {

typedef struct {
  int n_quads;
  const double* quads;  // [n_quads][9]  o, e1, e2
  int n_verts;
  const double* verts;  // [n_verts][3]
  const int* vert_h;    // [n_verts] height parameter index or -1
  int n_tris;
  const int* tris;      // [n_tris][3]
  const int* prim_mat;  // [n_quads + n_tris]
  int n_mats;
  const int* mat_type;  // 0 diffuse, 1 dielectric, 2 emitter
  const double* mat_ior;
  const int* mat_tex_off;
  const int* mat_tex_w;
  const int* mat_tex_h;
  int emitter_quad;
  double cam_pos[3], cam_look[3], cam_up[3];
  double fov_y_deg;
  int W, H;
} or_scene;

typedef struct {
  const double* albedo;
  int n_albedo;
  const double* Le;  // [3]
  const double* heights;
  int n_heights;
} or_params;

typedef struct {
  uint64_t seed;
  int64_t path_begin;  // first path index traced
  int64_t n_paths;     // number of paths traced
  int64_t n_norm;      // N in the 1/N estimator normalisation (total paths of the run)
  int max_depth;       // number of traced intersections x1..xD
  int method;          // see header comment
  int attached;        // 0 detached, 1 attached (geometry differentiated)
  int n_threads;
  int rr_depth;        // Russian roulette after vertices of depth >= rr_depth (0: off)
  double rr_q;         // its survival probability
  int filter;          // reconstruction filter: 0 tent (radius 1 px), 1 Gaussian (see filter_taps)
} or_run;

typedef struct {
  double* d_albedo;   // [n_albedo] or NULL
  double* d_Le;       // [3] or NULL
  double* d_heights;  // [n_heights] or NULL
  double* loss;       // [1] <dI, I_s> (or NULL)
} or_grads;
}

namespace {

const double PI = 3.14159265358979323846;
const double T_MIN = 1e-5;  // ray t lower bound (metres), also shadow-ray end margin

// ---------------------------------------------------------------- Philox4x32-10
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11):
// ten rounds of the 4x32 Philox bijection with multipliers 0xD2511F53, 0xCD9E8D57 and
// Weyl key increments 0x9E3779B9, 0xBB67AE85.
struct U4 { uint32_t v[4]; };
U4 philox(uint32_t k0, uint32_t k1, U4 c) {
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)0xD2511F53u * c.v[0];
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c.v[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    U4 o;
    o.v[0] = hi1 ^ c.v[1] ^ k0;
    o.v[1] = lo1;
    o.v[2] = hi0 ^ c.v[3] ^ k1;
    o.v[3] = lo0;
    c = o;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}
// Four uniforms in [0,1) for (path n, vertex depth d, stream s): 24-bit mantissas, exact
// in both float and double.
struct Rand4 { double u[4]; };
Rand4 rand4(uint64_t seed, uint64_t n, uint32_t d, uint32_t s) {
  U4 c = {{(uint32_t)n, (uint32_t)(n >> 32), d, s}};
  U4 o = philox((uint32_t)seed, (uint32_t)(seed >> 32), c);
  Rand4 r;
  for (int i = 0; i < 4; ++i) r.u[i] = (double)(o.v[i] >> 8) * (1.0 / 16777216.0);
  return r;
}

// ---------------------------------------------------------------- tape reverse-mode AD
struct Tape {
  std::vector<int> a, b;
  std::vector<double> da, db, adj;
  void clear() { a.clear(); b.clear(); da.clear(); db.clear(); }
  int push(int ia, double pa, int ib, double pb) {
    a.push_back(ia); da.push_back(pa); b.push_back(ib); db.push_back(pb);
    return (int)a.size() - 1;
  }
  void backward(int root) {
    adj.assign(a.size(), 0.0);
    adj[root] = 1.0;
    for (int i = (int)a.size() - 1; i >= 0; --i) {
      double g = adj[i];
      if (g == 0.0) continue;
      if (a[i] >= 0) adj[a[i]] += da[i] * g;
      if (b[i] >= 0) adj[b[i]] += db[i] * g;
    }
  }
};
thread_local Tape* TP = nullptr;

struct V {
  double v;
  int i;
  V() : v(0), i(-1) {}
  V(double x) : v(x), i(-1) {}
  V(double x, int id) : v(x), i(id) {}
};
inline V node(double v, int ia, double pa, int ib = -1, double pb = 0) {
  if (ia < 0 && ib < 0) return V(v);
  return V(v, TP->push(ia, pa, ib, pb));
}
inline V operator+(V x, V y) { return node(x.v + y.v, x.i, 1.0, y.i, 1.0); }
inline V operator-(V x, V y) { return node(x.v - y.v, x.i, 1.0, y.i, -1.0); }
inline V operator-(V x) { return node(-x.v, x.i, -1.0); }
inline V operator*(V x, V y) { return node(x.v * y.v, x.i, y.v, y.i, x.v); }
inline V operator/(V x, V y) { double q = x.v / y.v; return node(q, x.i, 1.0 / y.v, y.i, -q / y.v); }
inline V sqrt(V x) { double s = std::sqrt(x.v); return node(s, x.i, 0.5 / s); }
inline V fabs(V x) { return x.v < 0 ? -x : x; }
inline V expo(V x) { double e = std::exp(x.v); return node(e, x.i, e); }
inline double expo(double x) { return std::exp(x); }

inline double val(double x) { return x; }
inline double val(const V& x) { return x.v; }
using std::sqrt;
using std::fabs;

template <class T> struct Vec { T x, y, z; };
template <class T> Vec<T> mk(T x, T y, T z) { return Vec<T>{x, y, z}; }
template <class T> Vec<T> operator+(const Vec<T>& a, const Vec<T>& b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <class T> Vec<T> operator-(const Vec<T>& a, const Vec<T>& b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class T> Vec<T> operator*(const Vec<T>& a, T s) { return {a.x * s, a.y * s, a.z * s}; }
template <class T> T dot(const Vec<T>& a, const Vec<T>& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class T> Vec<T> cross(const Vec<T>& a, const Vec<T>& b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <class T> T norm(const Vec<T>& a) { return sqrt(dot(a, a)); }
template <class T> Vec<T> normalize(const Vec<T>& a) { T l = norm(a); return {a.x / l, a.y / l, a.z / l}; }
template <class T> Vec<double> vval(const Vec<T>& a) { return {val(a.x), val(a.y), val(a.z)}; }
template <class T> Vec<T> lift(const Vec<double>& a) { return {T(a.x), T(a.y), T(a.z)}; }
typedef Vec<double> D3;

// Orthonormal basis from a unit normal: Duff, Burgess, Christensen, Hery, Kensler,
// Liani, Villemin, "Building an Orthonormal Basis, Revisited" (JCGT 2017).
void onb(const D3& n, D3& t, D3& b) {
  double sign = std::copysign(1.0, n.z);
  double a = -1.0 / (sign + n.z);
  double bb = n.x * n.y * a;
  t = {1.0 + sign * n.x * n.x * a, sign * bb, -sign * n.x};
  b = {bb, sign + n.y * n.y * a, -n.y};
}

// ---------------------------------------------------------------- scene access
struct Scene {
  const or_scene* s;
  const or_params* p;
  int n_prims() const { return s->n_quads + s->n_tris; }
  int mat(int prim) const { return s->prim_mat[prim]; }
  int mtype(int prim) const { return s->mat_type[mat(prim)]; }
  // Camera frame and film constants (pinhole, image plane at distance 1).
  D3 cpos{}, cf{}, cr{}, cu{};
  double tanx = 0, tany = 0, A_img = 0;
  void setup() {
    cpos = {s->cam_pos[0], s->cam_pos[1], s->cam_pos[2]};
    D3 look = {s->cam_look[0], s->cam_look[1], s->cam_look[2]};
    D3 up = {s->cam_up[0], s->cam_up[1], s->cam_up[2]};
    cf = normalize(look - cpos);
    cr = normalize(cross(cf, up));
    cu = cross(cr, cf);
    tany = std::tan(0.5 * s->fov_y_deg * PI / 180.0);
    tanx = tany * (double)s->W / (double)s->H;
    A_img = 4.0 * tanx * tany;
  }
  // Primitive as o + s e1 + t e2.  Heights enter the triangle vertices' y coordinates.
  template <class T> void prim(int id, const T* heights, Vec<T>& o, Vec<T>& e1, Vec<T>& e2) const {
    if (id < s->n_quads) {
      const double* q = s->quads + 9 * id;
      o = mk<T>(q[0], q[1], q[2]); e1 = mk<T>(q[3], q[4], q[5]); e2 = mk<T>(q[6], q[7], q[8]);
      return;
    }
    const int* t = s->tris + 3 * (id - s->n_quads);
    Vec<T> v[3];
    for (int k = 0; k < 3; ++k) {
      const double* b = s->verts + 3 * t[k];
      v[k] = mk<T>(b[0], b[1], b[2]);
      int h = s->vert_h[t[k]];
      if (h >= 0) v[k].y = v[k].y + heights[h];
    }
    o = v[0]; e1 = v[1] - v[0]; e2 = v[2] - v[0];
  }
  bool is_quad(int id) const { return id < s->n_quads; }
};

// Moller & Trumbore, "Fast, minimum storage ray/triangle intersection" (1997), used for
// both triangles (s,t >= 0, s+t <= 1) and parallelograms (s,t in [0,1]).
bool hit_prim(const Scene& sc, int id, const double* hts, const D3& org, const D3& dir, double& t, double& su,
              double& sv) {
  D3 o, e1, e2;
  sc.prim<double>(id, hts, o, e1, e2);
  D3 pv = cross(dir, e2);
  double det = dot(e1, pv);
  if (det == 0.0) return false;
  double inv = 1.0 / det;
  D3 tv = org - o;
  double u = dot(tv, pv) * inv;
  D3 qv = cross(tv, e1);
  double v = dot(dir, qv) * inv;
  double tt = dot(e2, qv) * inv;
  if (sc.is_quad(id)) {
    if (u < 0.0 || u > 1.0 || v < 0.0 || v > 1.0) return false;
  } else {
    if (u < 0.0 || v < 0.0 || u + v > 1.0) return false;
  }
  t = tt; su = u; sv = v;
  return true;
}

// Closest hit by brute force over every primitive: smallest t > T_MIN, ties to the
// smaller primitive id, the primitive the ray leaves is skipped.
bool closest(const Scene& sc, const D3& org, const D3& dir, int skip, int& prim, double& t, double& su, double& sv) {
  prim = -1; t = 1e300;
  const double* h = sc.p->heights;
  for (int id = 0; id < sc.n_prims(); ++id) {
    if (id == skip) continue;
    double tt, u, v;
    if (hit_prim(sc, id, h, org, dir, tt, u, v) && tt > T_MIN && tt < t) { prim = id; t = tt; su = u; sv = v; }
  }
  return prim >= 0;
}
bool occluded(const Scene& sc, const D3& org, const D3& dir, double dist, int skip) {
  const double* h = sc.p->heights;
  for (int id = 0; id < sc.n_prims(); ++id) {
    if (id == skip) continue;
    double tt, u, v;
    if (hit_prim(sc, id, h, org, dir, tt, u, v) && tt > T_MIN && tt < dist - T_MIN) return true;
  }
  return false;
}

// Film projection (pixel units, row 0 at the top).  Returns false behind the camera.
template <class T> bool project(const Scene& sc, const Vec<T>& x, T& ux, T& uy, T& zc, T& dist) {
  Vec<T> d = x - lift<T>(sc.cpos);
  zc = dot(d, lift<T>(sc.cf));
  if (val(zc) <= 0) return false;
  dist = norm(d);
  T px = dot(d, lift<T>(sc.cr)) / zc, py = dot(d, lift<T>(sc.cu)) / zc;
  ux = T(0.5 * sc.s->W) * (T(1.0) + px / T(sc.tanx));
  uy = T(0.5 * sc.s->H) * (T(1.0) - py / T(sc.tany));
  return true;
}

// Smooth dielectric (Fresnel equations for unpolarised light).  `entering` when the ray
// arrives against the geometric normal.  Returns F and the two candidate directions.
template <class T> void dielectric(const Vec<T>& din, const Vec<T>& n, double ior, bool& entering, bool& tir, T& F,
                                   Vec<T>& refl, Vec<T>& refr) {
  entering = val(dot(din, n)) < 0;
  Vec<T> ns = entering ? n : n * T(-1.0);
  T eta = entering ? T(1.0 / ior) : T(ior);
  T ci = T(0.0) - dot(din, ns);
  refl = din + ns * (T(2.0) * ci);
  T s2t = eta * eta * (T(1.0) - ci * ci);
  tir = val(s2t) >= 1.0;
  if (tir) { F = T(1.0); refr = refl; return; }
  T ct = sqrt(T(1.0) - s2t);
  T rs = (eta * ci - ct) / (eta * ci + ct);
  T rp = (ci - eta * ct) / (ci + eta * ct);
  F = T(0.5) * (rs * rs + rp * rp);
  refr = din * eta + ns * (eta * ci - ct);
}

// Bilinear texture lookup with texel centres at (i+0.5)/w and clamp-to-edge.
template <class T> void texture(const Scene& sc, int m, const T* albedo, T s, T t, T rho[3]) {
  int w = sc.s->mat_tex_w[m], h = sc.s->mat_tex_h[m], off = sc.s->mat_tex_off[m];
  T tx = s * T((double)w) - T(0.5), ty = t * T((double)h) - T(0.5);
  double fx0 = std::floor(val(tx)), fy0 = std::floor(val(ty));
  T fx = tx - T(fx0), fy = ty - T(fy0);
  int x0 = (int)fx0, y0 = (int)fy0;
  int xa = std::min(std::max(x0, 0), w - 1), xb = std::min(std::max(x0 + 1, 0), w - 1);
  int ya = std::min(std::max(y0, 0), h - 1), yb = std::min(std::max(y0 + 1, 0), h - 1);
  T w00 = (T(1.0) - fx) * (T(1.0) - fy), w10 = fx * (T(1.0) - fy), w01 = (T(1.0) - fx) * fy, w11 = fx * fy;
  for (int c = 0; c < 3; ++c) {
    rho[c] = w00 * albedo[off + (ya * w + xa) * 3 + c] + w10 * albedo[off + (ya * w + xb) * 3 + c] +
             w01 * albedo[off + (yb * w + xa) * 3 + c] + w11 * albedo[off + (yb * w + xb) * 3 + c];
  }
}

inline double lum(const double L[3]) { return 0.2126 * L[0] + 0.7152 * L[1] + 0.0722 * L[2]; }

// ---------------------------------------------------------------- path decisions
enum { K_EMITTER = 0, K_DIFFUSE = 1, K_SPECULAR = 2 };
struct Vtx {
  int prim;
  bool attached;   // follows the emitter or a non-specular vertex
  double b1, b2;   // surface coordinates at the current parameters
  int kind;        // K_DIFFUSE or K_SPECULAR
  bool refl;       // specular branch
  bool conn;       // valid sensor connection (diffuse only)
  double g0 = -1;  // frozen value at theta0 of the attached segment weight G*A (or -1: not yet known)
  double F0 = -1;  // frozen value at theta0 of the chosen dielectric branch probability
  double rr = 1.0; // Russian-roulette weight 1/q applied after this vertex (1: none)
};
struct Path {
  D3 x0, n_light;
  std::vector<Vtx> v;
  int R = -1;       // reservoir winner (index into v) or -1
  double res_w = 0; // Omega_k / omega_R
  uint32_t hash = 2166136261u;
};
inline void fnv(uint32_t& h, uint32_t x) {  // FNV-1a over the four bytes of x
  for (int i = 0; i < 4; ++i) { h ^= (x >> (8 * i)) & 0xffu; h *= 16777619u; }
}

// Sensor connection test at a diffuse vertex: camera in the hemisphere the light arrived
// from, in front of the camera, on the film, and unoccluded (Sec. 3.1).
bool connect_ok(const Scene& sc, const D3& x, const D3& ns, int prim) {
  D3 c = sc.cpos - x;
  double dist = norm(c);
  D3 wc = c * (1.0 / dist);
  if (dot(ns, wc) <= 0) return false;
  double ux, uy, zc, dd;
  if (!project<double>(sc, x, ux, uy, zc, dd)) return false;
  if (!(ux >= 0 && ux < sc.s->W && uy >= 0 && uy < sc.s->H)) return false;
  return !occluded(sc, x, wc, dist, prim);
}


// Trace one light path at the current parameters and record every discrete decision
// (Sec. 3.1 light tracing: emitter sample, then intersect / connect / scatter per vertex).
// Uniforms: vertex depth d uses Philox counter (n, d, 0); at d=0 (emitter) u0,u1 pick the
// point on the light and u2,u3 a cosine-weighted direction; at d>=1 u0,u1 sample the
// diffuse direction, u2 the Fresnel branch, u3 the reservoir draw.  Russian roulette
// (rr_depth > 0): after the vertex of depth d >= rr_depth the path continues when the
// first uniform of Philox counter (n, d, 2) is below q, with weight 1/q; the decision
// does not depend on the parameters, so 1/q is a constant factor of the path function.
Path trace(const Scene& sc, uint64_t seed, uint64_t n, int D, int rr_depth, double rr_q) {
  Path P;
  const double* h = sc.p->heights;
  D3 lo, le1, le2;
  sc.prim<double>(sc.s->emitter_quad, h, lo, le1, le2);
  Rand4 r0 = rand4(seed, n, 0, 0);
  P.x0 = lo + le1 * r0.u[0] + le2 * r0.u[1];
  P.n_light = normalize(cross(le1, le2));
  D3 ta, tb;
  onb(P.n_light, ta, tb);
  double rr = std::sqrt(r0.u[2]), ph = 2 * PI * r0.u[3];
  D3 dir = ta * (rr * std::cos(ph)) + tb * (rr * std::sin(ph)) + P.n_light * std::sqrt(std::max(0.0, 1 - r0.u[2]));
  D3 org = P.x0;
  int skip = sc.s->emitter_quad;
  int prev = K_EMITTER;
  for (int d = 1; d <= D; ++d) {
    int prim;
    double tt, su, sv;
    if (!closest(sc, org, dir, skip, prim, tt, su, sv)) break;
    int mt = sc.mtype(prim);
    if (mt == 2) break;  // the emitter absorbs (its point x0 is never splatted)
    Vtx v;
    v.prim = prim; v.attached = (prev != K_SPECULAR); v.b1 = su; v.b2 = sv;
    v.refl = false; v.conn = false;
    D3 o, e1, e2;
    sc.prim<double>(prim, h, o, e1, e2);
    D3 x = v.attached ? o + e1 * su + e2 * sv : org + dir * tt;
    D3 nrm = normalize(cross(e1, e2));
    Rand4 r = rand4(seed, n, (uint32_t)d, 0);
    if (mt == 0) {
      v.kind = K_DIFFUSE;
      D3 ns = dot(nrm, dir) < 0 ? nrm : nrm * -1.0;
      v.conn = connect_ok(sc, x, ns, prim);
      onb(ns, ta, tb);
      double r1 = std::sqrt(r.u[0]), p1 = 2 * PI * r.u[1];
      dir = ta * (r1 * std::cos(p1)) + tb * (r1 * std::sin(p1)) + ns * std::sqrt(std::max(0.0, 1 - r.u[0]));
      prev = K_DIFFUSE;
    } else {
      v.kind = K_SPECULAR;
      bool ent, tir;
      double F;
      D3 rl, rf;
      dielectric<double>(dir, nrm, sc.s->mat_ior[sc.mat(prim)], ent, tir, F, rl, rf);
      v.refl = tir || r.u[2] < F;
      dir = v.refl ? rl : rf;
      prev = K_SPECULAR;
    }
    uint32_t flags = (uint32_t)v.kind | (v.refl ? 4u : 0u) | (v.conn ? 8u : 0u) | (v.attached ? 16u : 0u);
    fnv(P.hash, (uint32_t)prim);
    fnv(P.hash, flags);
    P.v.push_back(v);
    org = x;
    skip = prim;
    if (rr_depth > 0 && d >= rr_depth) {
      if (rand4(seed, n, (uint32_t)d, 2).u[0] < rr_q) P.v.back().rr = 1.0 / rr_q;
      else break;
    }
  }
  return P;
}

// Indexable parameter views: plain values, or lazily created AD leaves.
struct Plain {
  const double* a;
  double operator[](int i) const { return a[i]; }
};
struct ConstV {
  const double* a;
  V operator[](int i) const { return V(a[i]); }
};
struct Leaves {
  const double* a;
  std::vector<int>* node;     // param index -> tape node (-1 = none yet)
  std::vector<int>* touched;  // params with a node in the current tape
  V operator[](int i) const {
    int& id = (*node)[i];
    if (id < 0) { id = TP->push(-1, 0, -1, 0); touched->push_back(i); }
    return V(a[i], id);
  }
};

template <class T, class A> void prim_geom(const Scene& sc, int id, const A& hts, Vec<T>& o, Vec<T>& e1, Vec<T>& e2) {
  if (id < sc.s->n_quads) {
    const double* q = sc.s->quads + 9 * id;
    o = mk<T>(q[0], q[1], q[2]); e1 = mk<T>(q[3], q[4], q[5]); e2 = mk<T>(q[6], q[7], q[8]);
    return;
  }
  const int* t = sc.s->tris + 3 * (id - sc.s->n_quads);
  Vec<T> v[3];
  for (int k = 0; k < 3; ++k) {
    const double* b = sc.s->verts + 3 * t[k];
    v[k] = mk<T>(b[0], b[1], b[2]);
    int hh = sc.s->vert_h[t[k]];
    if (hh >= 0) v[k].y = v[k].y + hts[hh];
  }
  o = v[0]; e1 = v[1] - v[0]; e2 = v[2] - v[0];
}

template <class T, class A> void tex_lookup(const Scene& sc, int m, const A& albedo, T s, T t, T rho[3]) {
  int w = sc.s->mat_tex_w[m], h = sc.s->mat_tex_h[m], off = sc.s->mat_tex_off[m];
  T tx = s * T((double)w) - T(0.5), ty = t * T((double)h) - T(0.5);
  double fx0 = std::floor(val(tx)), fy0 = std::floor(val(ty));
  T fx = tx - T(fx0), fy = ty - T(fy0);
  int x0 = (int)fx0, y0 = (int)fy0;
  int xa = std::min(std::max(x0, 0), w - 1), xb = std::min(std::max(x0 + 1, 0), w - 1);
  int ya = std::min(std::max(y0, 0), h - 1), yb = std::min(std::max(y0 + 1, 0), h - 1);
  T w00 = (T(1.0) - fx) * (T(1.0) - fy), w10 = fx * (T(1.0) - fy), w01 = (T(1.0) - fx) * fy, w11 = fx * fy;
  for (int c = 0; c < 3; ++c)
    rho[c] = w00 * albedo[off + (ya * w + xa) * 3 + c] + w10 * albedo[off + (ya * w + xb) * 3 + c] +
             w01 * albedo[off + (yb * w + xa) * 3 + c] + w11 * albedo[off + (yb * w + xb) * 3 + c];
}

// Tent (bilinear) reconstruction filter of radius one pixel over pixel centres (i+0.5):
// the four taps around u.  Used identically for splatting and for the adjoint read.
template <class T> int tent_taps(int W, int H, T ux, T uy, int px[4], int py[4], T w[4]) {
  T gx = ux - T(0.5), gy = uy - T(0.5);
  double x0 = std::floor(val(gx)), y0 = std::floor(val(gy));
  T fx = gx - T(x0), fy = gy - T(y0);
  int ix = (int)x0, iy = (int)y0, k = 0;
  T wx[2] = {T(1.0) - fx, fx}, wy[2] = {T(1.0) - fy, fy};
  for (int j = 0; j < 2; ++j)
    for (int i = 0; i < 2; ++i) {
      int X = ix + i, Y = iy + j;
      if (X < 0 || X >= W || Y < 0 || Y >= H) continue;
      px[k] = X; py[k] = Y; w[k] = wx[i] * wy[j]; ++k;
    }
  return k;
}
// Wider filter (filter 1): separable truncated Gaussian of standard deviation 0.5 pixel
// over pixel centres, shifted down by its value at the radius 1.5 pixel so that it falls
// continuously to zero there, and normalised to unit integral per axis:
// g(d) = (exp(-2 d^2) - exp(-4.5)) / C for |d| < 1.5, C = sqrt(pi/2) erf(1.5 sqrt(2)) - 3 exp(-4.5).
// Up to three taps per axis.  filter 0 is the tent of tent_taps.
inline double gauss_norm() { return std::sqrt(PI / 2) * std::erf(1.5 * std::sqrt(2.0)) - 3.0 * std::exp(-4.5); }
template <class T> int filter_taps(int filter, int W, int H, T ux, T uy, int px[9], int py[9], T w[9]) {
  if (filter == 0) return tent_taps<T>(W, H, ux, uy, px, py, w);
  const double inv_c = 1.0 / gauss_norm(), cut = std::exp(-4.5);
  int xs[3], ys[3], nx = 0, ny = 0;
  T wx[3], wy[3];
  const double bx = std::floor(val(ux) - 0.5), by = std::floor(val(uy) - 0.5);
  for (int i = -1; i <= 2; ++i) {
    const int X = (int)bx + i;
    T dx = ux - T(X + 0.5);
    if (std::fabs(val(dx)) < 1.5 && X >= 0 && X < W && nx < 3) { xs[nx] = X; wx[nx] = (expo(T(-2.0) * dx * dx) - T(cut)) * T(inv_c); ++nx; }
    const int Y = (int)by + i;
    T dy = uy - T(Y + 0.5);
    if (std::fabs(val(dy)) < 1.5 && Y >= 0 && Y < H && ny < 3) { ys[ny] = Y; wy[ny] = (expo(T(-2.0) * dy * dy) - T(cut)) * T(inv_c); ++ny; }
  }
  int k = 0;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) { px[k] = xs[i]; py[k] = ys[j]; w[k] = wx[i] * wy[j]; ++k; }
  return k;
}

template <class T> void adjoint_read(const double* dI, int W, int H, T ux, T uy, T out[3], int filter) {
  int px[9], py[9];
  T w[9];
  int k = filter_taps<T>(filter, W, H, ux, uy, px, py, w);
  for (int c = 0; c < 3; ++c) {
    out[c] = T(0.0);
    for (int i = 0; i < k; ++i) out[c] = out[c] + w[i] * dI[(py[i] * W + px[i]) * 3 + c];
  }
}

template <class T> struct ConnOut {
  int vi;
  T L[3];
  T ux, uy;
  // values at the connection, for the per-connection query (or_connections): position,
  // arrival-side unit normal, arrival direction, throughput before the vertex's albedo and
  // the connection weight (importance with the estimator's 1/N)
  D3 x, ns, din;
  double beta[3], geo;
  // area density of the path's first vertex x1 as the light tracer samples it from x0
  // (cosine emission): cos0 cos1 / (pi r01^2); used by the bidirectional weights
  double pf0;
};

// Evaluate the frozen-decision path function: per valid sensor connection i, the splat
// L_i = W_e f_i G V (Eq. 1-2) and its film position u_i (Eq. 20), given the decisions in P.
// beta_0 = Le A_light pi (cosine emission from a uniformly sampled point); a diffuse
// vertex connects with f_s = rho/pi and importance  W H / (N A_img r^2 cos^3 theta_c)
// (pinhole, image plane at distance 1), then scatters with weight rho.
// lit_u: the film position of a connection at a sliding vertex is taken at the vertex's
// surface coordinates frozen at theta0 on its (moving) primitive, instead of at the
// position the specular chain delivers: the split used by the paper-literal attached
// variant (or_gradient_literal), whose chain transport of the film position is separate.
template <class T, class AA, class AL, class AH>
void eval_path(const Scene& sc, const Path& P, const AA& albedo, const AL& Le, const AH& hts, double N,
               std::vector<ConnOut<T>>& out, Path* fill = nullptr, bool lit_u = false) {
  // `fill`: evaluation at the decision parameters theta0; records the frozen denominators
  // (g0, F0) of the weight ratios so later evaluations at other parameters reuse them.
  out.clear();
  D3 lo, le1, le2;
  sc.prim<double>(sc.s->emitter_quad, sc.p->heights, lo, le1, le2);
  double A_L = norm(cross(le1, le2));
  T beta[3];
  for (int c = 0; c < 3; ++c) beta[c] = Le[c] * T(A_L * PI);
  Vec<T> xprev = lift<T>(P.x0), nprev = lift<T>(P.n_light), dprev = mk<T>(0.0, 0.0, 0.0);
  const double K = (double)sc.s->W * (double)sc.s->H / (sc.A_img * N * PI);
  double pf0 = 0.0;
  for (size_t k = 0; k < P.v.size(); ++k) {
    const Vtx& v = P.v[k];
    Vec<T> o, e1, e2;
    prim_geom<T>(sc, v.prim, hts, o, e1, e2);
    Vec<T> nraw = cross(e1, e2);
    T area = norm(nraw);
    Vec<T> n = nraw * (T(1.0) / area);
    Vec<T> x, din;
    T s, t;
    if (v.attached) {
      s = T(v.b1); t = T(v.b2);
      x = o + e1 * s + e2 * t;
      Vec<T> w = x - xprev;
      T r2 = dot(w, w);
      din = w * (T(1.0) / sqrt(r2));
      T g = fabs(dot(nprev, din)) * fabs(dot(n, din)) * area / r2;
      if (k == 0) pf0 = std::fabs(val(dot(nprev, din))) * std::fabs(val(dot(n, din))) / (PI * val(r2));
      if (fill) fill->v[k].g0 = val(g);
      T ratio = g / T(v.g0 > 0 ? v.g0 : val(g));
      for (int c = 0; c < 3; ++c) beta[c] = beta[c] * ratio;
    } else {
      din = dprev;
      T tt = dot(o - xprev, n) / dot(din, n);
      x = xprev + din * tt;
      Vec<T> q = x - o;
      T nn = dot(nraw, nraw);
      s = dot(cross(q, e2), nraw) / nn;
      t = dot(cross(e1, q), nraw) / nn;
    }
    int m = sc.mat(v.prim);
    if (v.kind == K_DIFFUSE) {
      T rho[3];
      tex_lookup<T>(sc, m, albedo, s, t, rho);
      Vec<T> ns = val(dot(n, din)) < 0 ? n : n * T(-1.0);
      if (v.conn) {
        Vec<T> cvec = lift<T>(sc.cpos) - x;
        T dist2 = dot(cvec, cvec);
        T dist = sqrt(dist2);
        T cosc = dot(ns, cvec) / dist;
        ConnOut<T> co;
        co.vi = (int)k;
        T zc, dd;
        project<T>(sc, x, co.ux, co.uy, zc, dd);
        if (lit_u && !v.attached) {
          T zl, dl;
          project<T>(sc, o + e1 * T(val(s)) + e2 * T(val(t)), co.ux, co.uy, zl, dl);
        }
        T cc = zc / dist;
        T geo = cosc * T(K) / (dist2 * cc * cc * cc);
        for (int c = 0; c < 3; ++c) co.L[c] = beta[c] * rho[c] * geo;
        co.x = vval(x); co.ns = vval(ns); co.din = vval(din);
        for (int c = 0; c < 3; ++c) co.beta[c] = val(beta[c]);
        co.geo = val(geo);
        co.pf0 = pf0;
        out.push_back(co);
      }
      for (int c = 0; c < 3; ++c) beta[c] = beta[c] * rho[c];
    } else {
      bool ent, tir;
      T F;
      Vec<T> rl, rf;
      dielectric<T>(din, n, sc.s->mat_ior[m], ent, tir, F, rl, rf);
      if (v.refl) {
        if (fill) fill->v[k].F0 = val(F);
        if (!tir) for (int c = 0; c < 3; ++c) beta[c] = beta[c] * (F / T(v.F0 > 0 ? v.F0 : val(F)));
        dprev = rl;
      } else {
        T omf = T(1.0) - F;
        if (fill) fill->v[k].F0 = val(omf);
        for (int c = 0; c < 3; ++c) beta[c] = beta[c] * (omf / T(v.F0 > 0 ? v.F0 : val(omf)));
        dprev = rf;
      }
    }
    if (v.rr != 1.0)
      for (int c = 0; c < 3; ++c) beta[c] = beta[c] * T(v.rr);
    xprev = x;
    nprev = n;
  }
}

// Weighted reservoir of capacity one over the valid connections (Sec. 4.2, Eq. 8):
// omega_i = luminance(L_i) (Rec. 709), Omega += omega_i, replace when u < omega_i/Omega.
// Connections with omega_i = 0 do not enter.  Returns R (index into `conns`) and Omega/omega_R.
int reservoir(const std::vector<double>& w, const std::vector<double>& u, double& res_w) {
  double Om = 0, wR = 0;
  int R = -1;
  for (size_t i = 0; i < w.size(); ++i) {
    if (!(w[i] > 0)) continue;
    Om += w[i];
    if (u[i] < w[i] / Om) { R = (int)i; wR = w[i]; }
  }
  res_w = R >= 0 ? Om / wR : 0.0;
  return R;
}

void path_reservoir(uint64_t seed, uint64_t n, Path& P, const std::vector<ConnOut<double>>& cs) {
  std::vector<double> w, u;
  for (auto& c : cs) {
    w.push_back(lum(c.L));
    u.push_back(rand4(seed, n, (uint32_t)(c.vi + 1), 0).u[3]);
  }
  double rw;
  int r = reservoir(w, u, rw);
  P.R = r;
  P.res_w = rw;
}

struct Ctx {
  const Scene* sc;
  const or_run* run;
  const double* dI;
  const uint8_t* mask;
};

// Per-thread accumulators.
struct Acc {
  std::vector<double> img, ga, gh;
  double gL[3] = {0, 0, 0};
  double loss = 0;
};

void splat(const Scene& sc, double* img, const double L[3], double ux, double uy, int filter) {
  int px[9], py[9];
  double w[9];
  int k = filter_taps<double>(filter, sc.s->W, sc.s->H, ux, uy, px, py, w);
  for (int i = 0; i < k; ++i)
    for (int c = 0; c < 3; ++c) img[(py[i] * sc.s->W + px[i]) * 3 + c] += w[i] * L[c];
}

template <class F> void parallel_paths(int n_threads, int64_t n, F&& f) {
  if (n_threads < 1) n_threads = 1;
  if (n_threads > n && n > 0) n_threads = (int)n;
  std::vector<std::thread> th;
  for (int t = 0; t < n_threads; ++t) {
    int64_t a = n * t / n_threads, b = n * (t + 1) / n_threads;
    th.emplace_back([&, t, a, b] { f(t, a, b); });
  }
  for (auto& x : th) x.join();
}

// Bilinear texel weights of a diffuse vertex (for the algorithm restatements).
void texel_weights(const Scene& sc, int m, double s, double t, int idx[4], double w[4]) {
  int tw = sc.s->mat_tex_w[m], th = sc.s->mat_tex_h[m], off = sc.s->mat_tex_off[m];
  double tx = s * tw - 0.5, ty = t * th - 0.5;
  double fx0 = std::floor(tx), fy0 = std::floor(ty), fx = tx - fx0, fy = ty - fy0;
  int x0 = (int)fx0, y0 = (int)fy0;
  int xa = std::min(std::max(x0, 0), tw - 1), xb = std::min(std::max(x0 + 1, 0), tw - 1);
  int ya = std::min(std::max(y0, 0), th - 1), yb = std::min(std::max(y0 + 1, 0), th - 1);
  idx[0] = off + (ya * tw + xa) * 3; w[0] = (1 - fx) * (1 - fy);
  idx[1] = off + (ya * tw + xb) * 3; w[1] = fx * (1 - fy);
  idx[2] = off + (yb * tw + xa) * 3; w[2] = (1 - fx) * fy;
  idx[3] = off + (yb * tw + xb) * 3; w[3] = fx * fy;
}

// ---------------------------------------------------------------- bidirectional estimator
// Two strategies for the same paths x0 (on the emitter), x1..xk (diffuse) -> camera, combined
// with the balance heuristic (Veach's multiple importance sampling):
//   L: a light path of the light tracer and its sensor connection at xk (N light paths);
//   C: a camera sample through a film position u uniform over the film, traced to
//      xk = y1, x_{k-1} = y2, ... by cosine sampling, with next-event estimation from
//      x1 = ym to a point x0 uniform on the emitter (M camera samples).
// With Lambertian surfaces, cosine sampling and cosine emission, the area densities of a
// segment between two surfaces are the same in both directions (cos cos / (pi r^2)), so
// the density ratio of C to L of a path reduces to
//   R = p_film(xk) / pf0,   p_film(xk) = cos_c / (A_img cos^3(theta_c) r_c^2),
//   pf0 = cos0 cos1 / (pi r01^2)  (x1 sampled from x0 by the light tracer),
// and either strategy's sample contributes  N L / (N + M R)  where L is the light tracer's
// splat value of the path (which carries 1/N): strategy L is weighted by N / (N + M R),
// strategy C by M R / (N + M R).  Diffuse scenes, detached, no Russian roulette.
struct CamVtx {
  int prim;
  double b1, b2;
  D3 x, ns;       // position and the unit normal on the side the camera path arrives from
  bool nee;       // valid next-event connection at this vertex
  D3 xl;          // its emitter point
};
struct CamPath {
  double ux, uy;
  std::vector<CamVtx> v;
  uint32_t hash = 2166136261u;
};

// Camera sample c: Philox stream 3, counter (c, 0) the film position, (c, m) at vertex m the
// cosine direction (u0, u1) and the emitter point of the next-event connection (u2, u3).
CamPath trace_cam(const Scene& sc, uint64_t seed, uint64_t c, int D) {
  CamPath P;
  const double* h = sc.p->heights;
  D3 lo, le1, le2;
  sc.prim<double>(sc.s->emitter_quad, h, lo, le1, le2);
  const D3 nL = normalize(cross(le1, le2));
  Rand4 r0 = rand4(seed, c, 0, 3);
  P.ux = r0.u[0] * sc.s->W;
  P.uy = r0.u[1] * sc.s->H;
  double pxn = (2 * P.ux / sc.s->W - 1) * sc.tanx, pyn = (1 - 2 * P.uy / sc.s->H) * sc.tany;
  D3 dir = normalize(sc.cf + sc.cr * pxn + sc.cu * pyn);
  D3 org = sc.cpos;
  int skip = -1;
  for (int m = 1; m <= D; ++m) {
    int prim;
    double tt, su, sv;
    if (!closest(sc, org, dir, skip, prim, tt, su, sv)) break;
    if (sc.mtype(prim) != 0) break;  // the emitter absorbs (seen directly it is black)
    CamVtx v;
    v.prim = prim; v.b1 = su; v.b2 = sv;
    D3 o, e1, e2;
    sc.prim<double>(prim, h, o, e1, e2);
    v.x = o + e1 * su + e2 * sv;
    D3 nrm = normalize(cross(e1, e2));
    v.ns = dot(nrm, dir) < 0 ? nrm : nrm * -1.0;
    Rand4 r = rand4(seed, c, (uint32_t)m, 3);
    v.xl = lo + le1 * r.u[2] + le2 * r.u[3];
    D3 wl = v.xl - v.x;
    double dist = norm(wl);
    D3 wn = wl * (1.0 / dist);
    v.nee = dot(v.ns, wn) > 0 && -dot(nL, wn) > 0 && !occluded(sc, v.x, wn, dist, prim);
    fnv(P.hash, (uint32_t)prim);
    fnv(P.hash, v.nee ? 1u : 0u);
    P.v.push_back(v);
    D3 ta, tb;
    onb(v.ns, ta, tb);
    double r1 = std::sqrt(r.u[0]), p1 = 2 * PI * r.u[1];
    dir = ta * (r1 * std::cos(p1)) + tb * (r1 * std::sin(p1)) + v.ns * std::sqrt(std::max(0.0, 1 - r.u[0]));
    org = v.x;
    skip = prim;
  }
  return P;
}

// Contribution of a camera sample, summed over its valid next-event connections (all splat
// at its film position): the connection at y_m closes the path x0 = xl, x1 = y_m, ...,
// xk = y_1 (k = m), whose light-tracer value times N is
//   Le A_L pi prod_{j=1..m} rho(y_j) geo(y_1),
// geo = cos_c W H / (A_img pi r_c^2 cos^3 theta_c) (the sensor connection at y_1); the
// sample adds it divided by (N + M R).  Values are evaluated with AD-capable albedo and Le.
template <class T, class AA, class AL>
void eval_cam(const Scene& sc, const CamPath& P, const AA& albedo, const AL& Le, double N, double M, T out[3]) {
  for (int c = 0; c < 3; ++c) out[c] = T(0.0);
  if (P.v.empty()) return;
  D3 lo, le1, le2;
  sc.prim<double>(sc.s->emitter_quad, sc.p->heights, lo, le1, le2);
  const D3 nL = normalize(cross(le1, le2));
  const double A_L = norm(cross(le1, le2));
  const D3 d = P.v[0].x - sc.cpos;
  const double dist = norm(d), cc = dot(d, sc.cf) / dist;
  const double cosc = -dot(P.v[0].ns, d) / dist;
  const double W = sc.s->W, H = sc.s->H;
  const double geo1 = cosc * W * H / (sc.A_img * PI * dist * dist * cc * cc * cc);
  const double pfilm = cosc / (sc.A_img * cc * cc * cc * dist * dist);
  T thr[3] = {T(1.0), T(1.0), T(1.0)};
  for (const CamVtx& v : P.v) {
    T rho[3];
    tex_lookup<T>(sc, sc.mat(v.prim), albedo, T(v.b1), T(v.b2), rho);
    for (int c = 0; c < 3; ++c) thr[c] = thr[c] * rho[c];
    if (!v.nee) continue;
    const D3 wl = v.xl - v.x;
    const double dl = norm(wl);
    const D3 wn = wl * (1.0 / dl);
    const double pf0 = dot(v.ns, wn) * -dot(nL, wn) / (PI * dl * dl);
    const double wgt = A_L * PI * geo1 / (N + M * (pfilm / pf0));
    for (int c = 0; c < 3; ++c) out[c] = out[c] + Le[c] * thr[c] * T(wgt);
  }
}

// Balance-heuristic weight N / (N + M R) of a light-tracer connection (see above).
double light_weight(const Scene& sc, const ConnOut<double>& c, double N, double M) {
  if (M <= 0) return 1.0;
  const double pfilm = c.geo * N * PI / ((double)sc.s->W * (double)sc.s->H);
  return N / (N + M * (pfilm / c.pf0));
}

// ---------------------------------------------------------------- paper-literal attached LRB-3
// The paper's attached formulation (Sec. 3.3, Eq. 4-7; Sec. 4.3.2, Eq. 18-19; Sec. 5) moves
// the splat-position adjoint along the path with forward-accumulated Jacobians of the
// two-point segment parameterisation p_j = (v_{j-1}, v_j) (v: surface coordinates, the
// emitter's (s, t) for j = 1): J_j = d p_{j+1} / d p_j (4x4), J_{1->j} = J_{j-1} ... J_1,
// A_pos = sum_i (0, 0, dL/du_i du_i/dv_i) J_{1->i} (Eq. 18, the position rows of the
// sensor Jacobian), and at vertex j the remainder projected back with the inverse,
// A_loc(j) = A_rem(j) J_{1->j}^{-1} (Eq. 19), replaced by zero when |det| falls below a
// threshold (Sec. 5) times the product of the row norms, or when a zero block has entered
// the product (singular by construction).  In this model a vertex that follows a diffuse vertex keeps its
// surface coordinates, so the lower block of J at a diffuse vertex is zero and J_{1->j}
// is singular after the first diffuse vertex: the guard then drops the transport along
// later (second-generation) specular chains.  Optional zero-mean noise (Sec. 5): at a
// diffuse vertex the lower block becomes eps sigma [I 0] with eps = +-1 from Philox stream 4
// at that depth (keyed by a noise seed of its own); the transport is linear in each noise
// factor, so it is unbiased over the noise.  The parameters enter the transport where a specular vertex maps p_j to p_{j+1}
// (K_j: the explicit dependence of v_{j+1} on the heights at fixed v_{j-1}, v_j), weighted
// by the position rows of A_loc(j+1).  Everything else (the radiance factors, each
// connection's film position at its own frozen surface coordinates) is the naive-AD
// gradient of the frozen path function with that split (eval_path's lit_u).

// Surface coordinates of the sliding vertex that follows specular vertex x_j (on prim j
// at v_j, reached from x_{j-1} on prim jp, or the emitter for jp = -1, at v_{j-1}) along the
// reflected (refl) or refracted direction, on prim jn's plane.
template <class T, class AH>
void spec_next(const Scene& sc, const AH& hts, int jp, const T vp[2], int j, const T vj[2], bool refl, int jn,
               T out[2]) {
  Vec<T> op, e1p, e2p;
  if (jp < 0) prim_geom<T>(sc, sc.s->emitter_quad, ConstV{sc.p->heights}, op, e1p, e2p);
  else prim_geom<T>(sc, jp, hts, op, e1p, e2p);
  Vec<T> o, e1, e2;
  prim_geom<T>(sc, j, hts, o, e1, e2);
  const Vec<T> xp = op + e1p * vp[0] + e2p * vp[1], xj = o + e1 * vj[0] + e2 * vj[1];
  const Vec<T> din = normalize(xj - xp);
  const Vec<T> n = normalize(cross(e1, e2));
  bool ent, tir;
  T F;
  Vec<T> rl, rf;
  dielectric<T>(din, n, sc.s->mat_ior[sc.mat(j)], ent, tir, F, rl, rf);
  const Vec<T> dout = refl ? rl : rf;
  Vec<T> on, e1n, e2n;
  prim_geom<T>(sc, jn, hts, on, e1n, e2n);
  const Vec<T> m = cross(e1n, e2n);
  const T tau = dot(on - xj, m) / dot(dout, m);
  const Vec<T> q = xj + dout * tau - on;
  const T nn = dot(m, m);
  out[0] = dot(cross(q, e2n), m) / nn;
  out[1] = dot(cross(e1n, q), m) / nn;
}

typedef double M4[4][4];
void m4_mul(const M4 a, const M4 b, M4 c) {  // c = a b
  M4 r;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      r[i][j] = 0;
      for (int k = 0; k < 4; ++k) r[i][j] += a[i][k] * b[k][j];
    }
  std::memcpy(c, r, sizeof(M4));
}
// Inverse by Gauss-Jordan elimination with partial pivoting; false when |det| < eps times
// the product of the row norms (Hadamard's bound on |det|: a scale-free test of singularity).
bool m4_inv(const M4 a, M4 inv, double eps) {
  double bound = 1.0;
  for (int i = 0; i < 4; ++i)
    bound *= std::sqrt(a[i][0] * a[i][0] + a[i][1] * a[i][1] + a[i][2] * a[i][2] + a[i][3] * a[i][3]);
  if (!(bound > 0.0)) return false;
  double m[4][8];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 8; ++j) m[i][j] = j < 4 ? a[i][j] : (j - 4 == i ? 1.0 : 0.0);
  double det = 1.0;
  for (int c = 0; c < 4; ++c) {
    int pr = c;
    for (int r = c + 1; r < 4; ++r)
      if (std::fabs(m[r][c]) > std::fabs(m[pr][c])) pr = r;
    if (pr != c) {
      for (int j = 0; j < 8; ++j) std::swap(m[pr][j], m[c][j]);
      det = -det;
    }
    det *= m[c][c];
    if (m[c][c] == 0.0) return false;
    for (int r = 0; r < 4; ++r) {
      if (r == c) continue;
      const double f = m[r][c] / m[c][c];
      for (int j = 0; j < 8; ++j) m[r][j] -= f * m[c][j];
    }
  }
  if (!(std::fabs(det) >= eps * bound)) return false;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) inv[i][j] = m[i][j + 4] / m[i][i];
  return true;
}

int bidir_check(const or_scene* s, const or_run* run) {
  if (run->attached) return -1;
  for (int m = 0; m < s->n_mats; ++m)
    if (s->mat_type[m] == 1) return -2;
  if (run->rr_depth > 0) return -3;
  return 0;
}

}  // namespace

// =============================================================================== C API
extern "C" {

// One Philox4x32-10 block (Salmon et al., SC'11): the counter-based generator every pass
// replays from (Sec. 3.2: a path is regenerated from its seed, not stored).
void or_philox(uint32_t k0, uint32_t k1, const uint32_t* ctr, uint32_t* out) {
  U4 c = {{ctr[0], ctr[1], ctr[2], ctr[3]}};
  U4 o = philox(k0, k1, c);
  for (int i = 0; i < 4; ++i) out[i] = o.v[i];
}

// Taps of the reconstruction filter at film position (ux, uy): pixel coordinates and
// weights (at most 9); returns their count.
int or_filter_taps(int filter, int W, int H, double ux, double uy, int* px, int* py, double* w) {
  return filter_taps<double>(filter, W, H, ux, uy, px, py, w);
}

// The four uniforms in [0, 1) of path n at vertex depth d from Philox stream s (the
// counter layout both sides implement from the generator's definition).
void or_uniforms(uint64_t seed, uint64_t n, uint32_t d, uint32_t s, double* out4) {
  Rand4 r = rand4(seed, n, d, s);
  for (int i = 0; i < 4; ++i) out4[i] = r.u[i];
}

// Smooth-dielectric scattering of a unit direction at a surface with geometric normal n:
// unpolarised Fresnel reflectance, Snell refraction, total internal reflection; the
// branch is chosen by u against F (the BSDF sampling step of Eq. 2's throughput).
void or_dielectric(const double* din, const double* n, double ior, double u, double* dout, double* F, int* refl) {
  D3 d = {din[0], din[1], din[2]}, nn = {n[0], n[1], n[2]}, rl, rf;
  bool ent, tir;
  double f;
  dielectric<double>(d, nn, ior, ent, tir, f, rl, rf);
  bool r = tir || u < f;
  D3 o = r ? rl : rf;
  dout[0] = o.x; dout[1] = o.y; dout[2] = o.z;
  *F = f;
  *refl = r ? 1 : 0;
}

// Capacity-one weighted reservoir over candidate weights w with uniforms u (Sec. 4.2,
// Eq. 8-9): the selected index (or -1) and Omega / omega_R.
int or_reservoir(const double* w, int n, const double* u, double* res_w) {
  std::vector<double> ww(w, w + n), uu(u, u + n);
  return reservoir(ww, uu, *res_w);
}

// Closest hit from org along dir (skipping primitive `skip`) by testing every primitive
// (no acceleration structure); returns the primitive or -1.
int or_intersect(const or_scene* s, const or_params* p, const double* org, const double* dir, int skip, double* out3) {
  Scene sc{s, p};
  sc.setup();
  int prim;
  double t, su, sv;
  if (!closest(sc, {org[0], org[1], org[2]}, {dir[0], dir[1], dir[2]}, skip, prim, t, su, sv)) return -1;
  out3[0] = t; out3[1] = su; out3[2] = sv;
  return prim;
}

// Light-traced image (Sec. 3.1).  estimator 0 splats every connection; estimator 1 splats
// only the reservoir winner reweighted by Omega/omega_R (Eq. 9, the ResLRB primal);
// estimator 2 returns the tap-mass image used to bound film-position rounding; estimator 3
// splats every connection like 0 and reports per path the smallest distance (pixels) of a
// film coordinate of its connections to a pixel centre, where the tent filter's derivative
// jumps (Eq. 21; 1e9 without connections).  image [H][W][3] is overwritten.  Optional
// per-path outputs: hashes [n_paths], records [n_paths][8] = (R vertex index or -1,
// Omega/omega_R, u_x, u_y, S_rgb, n_conn); estimator 3: records [n_paths][8] with the
// distance in slot 0.
int or_render_lt(const or_scene* s, const or_params* p, const or_run* run, const uint8_t* mask, double* image,
                 uint32_t* hashes, int estimator, double* records) {
  Scene sc{s, p};
  sc.setup();
  const int64_t npx = (int64_t)s->W * s->H * 3;
  int nt = std::max(1, run->n_threads);
  std::vector<Acc> acc(nt);
  const double N = (double)(run->n_norm > 0 ? run->n_norm : run->n_paths);
  parallel_paths(nt, run->n_paths, [&](int tid, int64_t a, int64_t b) {
    Acc& A = acc[tid];
    A.img.assign(npx, 0.0);
    std::vector<ConnOut<double>> cs;
    for (int64_t i = a; i < b; ++i) {
      uint64_t n = (uint64_t)(run->path_begin + i);
      Path P = trace(sc, run->seed, n, run->max_depth, run->rr_depth, run->rr_q);
      if (hashes) hashes[i] = P.hash;
      eval_path<double>(sc, P, Plain{p->albedo}, Plain{p->Le}, Plain{p->heights}, N, cs, &P);
      if (records) {
        double* r = records + 8 * i;
        for (int k = 0; k < 8; ++k) r[k] = 0;
        r[0] = -1;
        r[7] = (double)cs.size();
      }
      if (estimator == 3 && records) {
        double dmin = 1e9;
        for (auto& c : cs)
          for (double u : {c.ux, c.uy}) dmin = std::min(dmin, std::fabs((u - 0.5) - std::round(u - 0.5)));
        records[8 * i] = dmin;
      }
      if (mask && !mask[i]) continue;
      if (estimator == 0 || estimator == 3) {
        for (auto& c : cs) splat(sc, A.img.data(), c.L, c.ux, c.uy, run->filter);
      } else if (estimator == 2) {
        // tap mass: |L| added with weight one to every on-film tap of each splat (bounds
        // how much a film-position error can move a pixel)
        for (auto& c : cs) {
          int px[9], py[9];
          double w[9];
          int k = filter_taps<double>(run->filter, sc.s->W, sc.s->H, c.ux, c.uy, px, py, w);
          for (int t = 0; t < k; ++t)
            for (int ch = 0; ch < 3; ++ch) A.img[(py[t] * sc.s->W + px[t]) * 3 + ch] += std::fabs(c.L[ch]);
        }
      } else {
        path_reservoir(run->seed, n, P, cs);
        if (P.R < 0) continue;
        const ConnOut<double>& c = cs[P.R];
        double S[3] = {c.L[0] * P.res_w, c.L[1] * P.res_w, c.L[2] * P.res_w};
        splat(sc, A.img.data(), S, c.ux, c.uy, run->filter);
        if (records) {
          double* r = records + 8 * i;
          r[0] = c.vi; r[1] = P.res_w; r[2] = c.ux; r[3] = c.uy;
          r[4] = S[0]; r[5] = S[1]; r[6] = S[2];
        }
      }
    }
  });
  for (int64_t j = 0; j < npx; ++j) {
    double v = 0;
    for (int t = 0; t < nt; ++t) v += acc[t].img.size() ? acc[t].img[j] : 0.0;
    image[j] = v;
  }
  return 0;
}

// Gradient of <dI, I_s(theta)> (see header for methods: naive AD, Sec. 3.2; LRB-3-pass,
// Sec. 4.3, Eq. 14-19; ResLRB, Sec. 4.2, Eq. 9-13).  Outputs are overwritten.
// path_dbg (optional) [n_paths][4] = (delta_total rgb, number of valid connections).
int or_gradient(const or_scene* s, const or_params* p, const or_run* run, const double* dI, const uint8_t* mask,
                or_grads* out, uint32_t* hashes, double* path_dbg) {
  Scene sc{s, p};
  sc.setup();
  if (run->method == 1 || run->method == 3) {  // restatements: detached, all-diffuse scenes only
    if (run->attached) return -1;
    for (int m = 0; m < s->n_mats; ++m)
      if (s->mat_type[m] == 1) return -2;
  }
  int nt = std::max(1, run->n_threads);
  std::vector<Acc> acc(nt);
  const double N = (double)(run->n_norm > 0 ? run->n_norm : run->n_paths);
  const int W = s->W, H = s->H;
  parallel_paths(nt, run->n_paths, [&](int tid, int64_t a, int64_t b) {
    Acc& A = acc[tid];
    A.ga.assign(p->n_albedo, 0.0);
    A.gh.assign(p->n_heights, 0.0);
    Tape tape;
    TP = &tape;
    std::vector<int> node_a(p->n_albedo, -1), node_h(p->n_heights, -1), touch_a, touch_h;
    std::vector<ConnOut<double>> cs;
    std::vector<ConnOut<V>> cv;
    for (int64_t i = a; i < b; ++i) {
      uint64_t n = (uint64_t)(run->path_begin + i);
      Path P = trace(sc, run->seed, n, run->max_depth, run->rr_depth, run->rr_q);
      if (hashes) hashes[i] = P.hash;
      eval_path<double>(sc, P, Plain{p->albedo}, Plain{p->Le}, Plain{p->heights}, N, cs, &P);
      double dt[3] = {0, 0, 0};
      for (auto& c : cs) {
        double Lb[3];
        adjoint_read<double>(dI, W, H, c.ux, c.uy, Lb, run->filter);
        for (int k = 0; k < 3; ++k) dt[k] += Lb[k] * c.L[k];
      }
      if (path_dbg) {
        double* r = path_dbg + 4 * i;
        r[0] = dt[0]; r[1] = dt[1]; r[2] = dt[2]; r[3] = (double)cs.size();
      }
      if (mask && !mask[i]) continue;
      if (run->method == 2 || run->method == 3) path_reservoir(run->seed, n, P, cs);
      if (run->method == 0 || run->method == 2) {
        // naive reverse-mode AD over the whole path (tape grows with path length)
        if (run->method == 2 && P.R < 0) continue;
        tape.clear();
        touch_a.clear(); touch_h.clear();
        V Lev[3];
        for (int c = 0; c < 3; ++c) Lev[c] = V(p->Le[c], tape.push(-1, 0, -1, 0));
        Leaves la{p->albedo, &node_a, &touch_a};
        if (run->attached) {
          Leaves lh{p->heights, &node_h, &touch_h};
          eval_path<V>(sc, P, la, Lev, lh, N, cv);
        } else {
          eval_path<V>(sc, P, la, Lev, ConstV{p->heights}, N, cv);
        }
        V loss(0.0);
        for (size_t j = 0; j < cv.size(); ++j) {
          if (run->method == 2 && (int)j != P.R) continue;
          V Lb[3];
          adjoint_read<V>(dI, W, H, cv[j].ux, cv[j].uy, Lb, run->filter);
          V term = cv[j].L[0] * Lb[0] + cv[j].L[1] * Lb[1] + cv[j].L[2] * Lb[2];
          if (run->method == 2) term = term * V(P.res_w);
          loss = loss + term;
        }
        A.loss += loss.v;
        if (loss.i >= 0) {
          tape.backward(loss.i);
          for (int c = 0; c < 3; ++c) A.gL[c] += tape.adj[Lev[c].i];
          for (int idx : touch_a) A.ga[idx] += tape.adj[node_a[idx]];
          for (int idx : touch_h) A.gh[idx] += tape.adj[node_h[idx]];
        }
        for (int idx : touch_a) node_a[idx] = -1;
        for (int idx : touch_h) node_h[idx] = -1;
      } else {
        // Algorithm restatements (detached).  Per valid connection i: P_i = Lbar_i * L_i.
        // LRB-3-pass: pass 2 sums delta_total = sum_i P_i (Eq. 14); pass 3 walks the
        // vertices again, backpropagates the splat factor with P_i (Eq. 15), subtracts
        // P_i from delta_rem (Eq. 16) and backpropagates the scattering factor with the
        // remaining adjoint delta_rem (Eq. 17).  ResLRB: one connection R with weight
        // P = Lbar_R * S (Eq. 11) applied to every factor up to R.
        std::vector<double> Pw(3 * cs.size());
        for (size_t j = 0; j < cs.size(); ++j) {
          double Lb[3];
          adjoint_read<double>(dI, W, H, cs[j].ux, cs[j].uy, Lb, run->filter);
          for (int c = 0; c < 3; ++c) Pw[3 * j + c] = Lb[c] * cs[j].L[c];
        }
        double rem[3];
        int last = (int)P.v.size() - 1;
        if (run->method == 1) {
          for (int c = 0; c < 3; ++c) { rem[c] = dt[c]; A.gL[c] += dt[c] / p->Le[c]; A.loss += dt[c]; }
        } else {
          if (P.R < 0) continue;
          for (int c = 0; c < 3; ++c) { rem[c] = Pw[3 * P.R + c] * P.res_w; A.gL[c] += rem[c] / p->Le[c]; A.loss += rem[c]; }
          last = cs[P.R].vi;
        }
        size_t ci = 0;
        for (int k = 0; k <= last; ++k) {
          const Vtx& v = P.v[k];
          if (v.kind != K_DIFFUSE) continue;
          int m = sc.mat(v.prim);
          int idx[4];
          double tw[4], rho[3];
          texel_weights(sc, m, v.b1, v.b2, idx, tw);  // every vertex is attached in an all-diffuse scene
          tex_lookup<double>(sc, m, Plain{p->albedo}, v.b1, v.b2, rho);
          double wsplat[3] = {0, 0, 0};
          bool has = ci < cs.size() && cs[ci].vi == k;
          if (has) {
            if (run->method == 1) {
              for (int c = 0; c < 3; ++c) { wsplat[c] = Pw[3 * ci + c]; rem[c] -= Pw[3 * ci + c]; }
            } else if ((int)ci == P.R) {
              for (int c = 0; c < 3; ++c) wsplat[c] = rem[c];
            }
            ++ci;
          }
          bool scatter = run->method == 1 ? true : (k < last);
          for (int c = 0; c < 3; ++c) {
            double wt = wsplat[c] + (scatter ? rem[c] : 0.0);
            for (int q = 0; q < 4; ++q) A.ga[idx[q] + c] += wt / rho[c] * tw[q];
          }
        }
      }
    }
    TP = nullptr;
  });
  if (out->d_albedo) for (int j = 0; j < p->n_albedo; ++j) { double v = 0; for (int t = 0; t < nt; ++t) if (acc[t].ga.size()) v += acc[t].ga[j]; out->d_albedo[j] = v; }
  if (out->d_heights) for (int j = 0; j < p->n_heights; ++j) { double v = 0; for (int t = 0; t < nt; ++t) if (acc[t].gh.size()) v += acc[t].gh[j]; out->d_heights[j] = v; }
  if (out->d_Le) for (int c = 0; c < 3; ++c) { double v = 0; for (int t = 0; t < nt; ++t) v += acc[t].gL[c]; out->d_Le[c] = v; }
  if (out->loss) { double v = 0; for (int t = 0; t < nt; ++t) v += acc[t].loss; out->loss[0] = v; }
  return 0;
}

// Every valid sensor connection of the paths (in path order, skipping masked paths), one
// row of 24 doubles each: path index, vertex index k (depth k+1), position x[3], arrival-side
// unit normal[3], unit arrival direction[3], throughput before the vertex's albedo[3], film
// position u_x, u_y, connection weight (importance including the estimator's 1/N), the
// splat L[3] (Eq. 1) and its filter-weighted adjoint read Lbar[3] (Eq. 21), 0.  At most
// `cap` rows are written; returns the number of connections.
int64_t or_connections(const or_scene* s, const or_params* p, const or_run* run, const double* dI,
                       const uint8_t* mask, double* rows, int64_t cap) {
  Scene sc{s, p};
  sc.setup();
  const double N = (double)(run->n_norm > 0 ? run->n_norm : run->n_paths);
  std::vector<ConnOut<double>> cs;
  int64_t count = 0;
  for (int64_t i = 0; i < run->n_paths; ++i) {
    if (mask && !mask[i]) continue;
    uint64_t n = (uint64_t)(run->path_begin + i);
    Path P = trace(sc, run->seed, n, run->max_depth, run->rr_depth, run->rr_q);
    eval_path<double>(sc, P, Plain{p->albedo}, Plain{p->Le}, Plain{p->heights}, N, cs, &P);
    for (auto& c : cs) {
      if (count < cap) {
        double* r = rows + 24 * count;
        double Lb[3];
        adjoint_read<double>(dI, s->W, s->H, c.ux, c.uy, Lb, run->filter);
        const double v[24] = {(double)i, (double)c.vi, c.x.x, c.x.y, c.x.z, c.ns.x, c.ns.y, c.ns.z,
                              c.din.x, c.din.y, c.din.z, c.beta[0], c.beta[1], c.beta[2], c.ux, c.uy, c.geo,
                              c.L[0], c.L[1], c.L[2], Lb[0], Lb[1], Lb[2], 0.0};
        for (int k = 0; k < 24; ++k) r[k] = v[k];
      }
      ++count;
    }
  }
  return count;
}

// <dI, I_s> with every decision taken at parameters p0 and every value evaluated at p1
// (the frozen-decision function whose derivative all methods compute).  method 0: all
// connections; method 2: the ResLRB estimator (winner and weight frozen at p0).
double or_frozen_loss(const or_scene* s, const or_params* p0, const or_params* p1, const or_run* run,
                      const double* dI, const uint8_t* mask) {
  Scene sc0{s, p0};
  sc0.setup();
  Scene sc1{s, p1};
  sc1.setup();
  int nt = std::max(1, run->n_threads);
  std::vector<double> part(nt, 0.0);
  const double N = (double)(run->n_norm > 0 ? run->n_norm : run->n_paths);
  parallel_paths(nt, run->n_paths, [&](int tid, int64_t a, int64_t b) {
    std::vector<ConnOut<double>> cs;
    for (int64_t i = a; i < b; ++i) {
      if (mask && !mask[i]) continue;
      uint64_t n = (uint64_t)(run->path_begin + i);
      Path P = trace(sc0, run->seed, n, run->max_depth, run->rr_depth, run->rr_q);
      eval_path<double>(sc0, P, Plain{p0->albedo}, Plain{p0->Le}, Plain{p0->heights}, N, cs, &P);
      if (run->method == 2) {
        path_reservoir(run->seed, n, P, cs);
        if (P.R < 0) continue;
      }
      eval_path<double>(sc1, P, Plain{p1->albedo}, Plain{p1->Le}, Plain{p1->heights}, N, cs);
      for (size_t j = 0; j < cs.size(); ++j) {
        if (run->method == 2 && (int)j != P.R) continue;
        double Lb[3];
        adjoint_read<double>(dI, s->W, s->H, cs[j].ux, cs[j].uy, Lb, run->filter);
        double term = cs[j].L[0] * Lb[0] + cs[j].L[1] * Lb[1] + cs[j].L[2] * Lb[2];
        part[tid] += run->method == 2 ? term * P.res_w : term;
      }
    }
  });
  double v = 0;
  for (double x : part) v += x;
  return v;
}

// Bidirectional estimator (Discussion, "Toward more complex integrators": light tracer +
// camera samples with next-event estimation, balance heuristic; see above): image [H][W][3] overwritten.  N = run->n_norm (or
// n_paths) light paths from run, n_cam camera samples (indices 0..n_cam-1).  Optional
// per-sample decision hashes of the light paths (hashes [n_paths]) and camera samples
// (cam_hashes [n_cam]); masks skip paths / samples.  Returns < 0 for unsupported requests
// (attached, dielectrics, Russian roulette).
int or_render_bidir(const or_scene* s, const or_params* p, const or_run* run, int64_t n_cam, const uint8_t* mask,
                    const uint8_t* cam_mask, double* image, uint32_t* hashes, uint32_t* cam_hashes) {
  const int bad = bidir_check(s, run);
  if (bad) return bad;
  Scene sc{s, p};
  sc.setup();
  const int64_t npx = (int64_t)s->W * s->H * 3;
  const double N = (double)(run->n_norm > 0 ? run->n_norm : run->n_paths), M = (double)n_cam;
  int nt = std::max(1, run->n_threads);
  std::vector<Acc> acc(nt);
  parallel_paths(nt, run->n_paths, [&](int tid, int64_t a, int64_t b) {
    Acc& A = acc[tid];
    A.img.assign(npx, 0.0);
    std::vector<ConnOut<double>> cs;
    for (int64_t i = a; i < b; ++i) {
      uint64_t n = (uint64_t)(run->path_begin + i);
      Path P = trace(sc, run->seed, n, run->max_depth, 0, 1.0);
      if (hashes) hashes[i] = P.hash;
      if (mask && !mask[i]) continue;
      eval_path<double>(sc, P, Plain{p->albedo}, Plain{p->Le}, Plain{p->heights}, N > 0 ? N : 1.0, cs, &P);
      for (auto& c : cs) {
        const double w = light_weight(sc, c, N, M);
        double L[3] = {c.L[0] * w, c.L[1] * w, c.L[2] * w};
        splat(sc, A.img.data(), L, c.ux, c.uy, run->filter);
      }
    }
  });
  std::vector<Acc> cacc(nt);
  parallel_paths(nt, n_cam, [&](int tid, int64_t a, int64_t b) {
    Acc& A = cacc[tid];
    A.img.assign(npx, 0.0);
    for (int64_t c = a; c < b; ++c) {
      CamPath P = trace_cam(sc, run->seed, (uint64_t)c, run->max_depth);
      if (cam_hashes) cam_hashes[c] = P.hash;
      if (cam_mask && !cam_mask[c]) continue;
      double L[3];
      eval_cam<double>(sc, P, Plain{p->albedo}, Plain{p->Le}, N, M, L);
      splat(sc, A.img.data(), L, P.ux, P.uy, run->filter);
    }
  });
  for (int64_t j = 0; j < npx; ++j) {
    double v = 0;
    for (int t = 0; t < nt; ++t) {
      v += acc[t].img.size() ? acc[t].img[j] : 0.0;
      v += cacc[t].img.size() ? cacc[t].img[j] : 0.0;
    }
    image[j] = v;
  }
  return 0;
}

// Naive reverse-mode AD (tape per light path and per camera sample) of <dI, I_bidir> for
// the bidirectional estimator of or_render_bidir: albedo and Le gradients (detached; the
// balance-heuristic weights depend on the geometry only).  Outputs are overwritten.
int or_gradient_bidir(const or_scene* s, const or_params* p, const or_run* run, int64_t n_cam, const double* dI,
                      const uint8_t* mask, const uint8_t* cam_mask, or_grads* out) {
  const int bad = bidir_check(s, run);
  if (bad) return bad;
  Scene sc{s, p};
  sc.setup();
  const double N = (double)(run->n_norm > 0 ? run->n_norm : run->n_paths), M = (double)n_cam;
  const int W = s->W, H = s->H;
  int nt = std::max(1, run->n_threads);
  std::vector<Acc> acc(nt);
  auto body = [&](int tid, int64_t a, int64_t b, bool camera) {
    Acc& A = acc[tid];
    if (A.ga.empty()) A.ga.assign(p->n_albedo, 0.0);
    Tape tape;
    TP = &tape;
    std::vector<int> node_a(p->n_albedo, -1), touch_a;
    std::vector<ConnOut<double>> cs;
    std::vector<ConnOut<V>> cv;
    for (int64_t i = a; i < b; ++i) {
      tape.clear();
      touch_a.clear();
      V Lev[3];
      for (int c = 0; c < 3; ++c) Lev[c] = V(p->Le[c], tape.push(-1, 0, -1, 0));
      Leaves la{p->albedo, &node_a, &touch_a};
      V loss(0.0);
      if (camera) {
        if (cam_mask && !cam_mask[i]) continue;
        CamPath P = trace_cam(sc, run->seed, (uint64_t)i, run->max_depth);
        V L[3];
        eval_cam<V>(sc, P, la, Lev, N, M, L);
        double Lb[3];
        adjoint_read<double>(dI, W, H, P.ux, P.uy, Lb, run->filter);
        for (int c = 0; c < 3; ++c) loss = loss + L[c] * V(Lb[c]);
      } else {
        if (mask && !mask[i]) continue;
        uint64_t n = (uint64_t)(run->path_begin + i);
        Path P = trace(sc, run->seed, n, run->max_depth, 0, 1.0);
        eval_path<double>(sc, P, Plain{p->albedo}, Plain{p->Le}, Plain{p->heights}, N > 0 ? N : 1.0, cs, &P);
        eval_path<V>(sc, P, la, Lev, ConstV{p->heights}, N > 0 ? N : 1.0, cv);
        for (size_t j = 0; j < cv.size(); ++j) {
          const double w = light_weight(sc, cs[j], N, M);
          V Lb[3];
          adjoint_read<V>(dI, W, H, cv[j].ux, cv[j].uy, Lb, run->filter);
          V term = cv[j].L[0] * Lb[0] + cv[j].L[1] * Lb[1] + cv[j].L[2] * Lb[2];
          loss = loss + term * V(w);
        }
      }
      A.loss += loss.v;
      if (loss.i >= 0) {
        tape.backward(loss.i);
        for (int c = 0; c < 3; ++c) A.gL[c] += tape.adj[Lev[c].i];
        for (int idx : touch_a) A.ga[idx] += tape.adj[node_a[idx]];
      }
      for (int idx : touch_a) node_a[idx] = -1;
    }
    TP = nullptr;
  };
  parallel_paths(nt, run->n_paths, [&](int tid, int64_t a, int64_t b) { body(tid, a, b, false); });
  parallel_paths(nt, n_cam, [&](int tid, int64_t a, int64_t b) { body(tid, a, b, true); });
  if (out->d_albedo)
    for (int j = 0; j < p->n_albedo; ++j) {
      double v = 0;
      for (int t = 0; t < nt; ++t) if (acc[t].ga.size()) v += acc[t].ga[j];
      out->d_albedo[j] = v;
    }
  if (out->d_heights) for (int j = 0; j < p->n_heights; ++j) out->d_heights[j] = 0.0;
  if (out->d_Le) for (int c = 0; c < 3; ++c) { double v = 0; for (int t = 0; t < nt; ++t) v += acc[t].gL[c]; out->d_Le[c] = v; }
  if (out->loss) { double v = 0; for (int t = 0; t < nt; ++t) v += acc[t].loss; out->loss[0] = v; }
  return 0;
}

// Paper-literal attached LRB-3 gradient of <dI, I_s> (Eq. 4-7, Eq. 18-19, Sec. 5; see the
// section above): naive AD of
// the frozen path function with each connection's film position at its own frozen surface
// coordinates, plus the film-position transport along specular chains by accumulated
// two-point Jacobians with the determinant-guarded inverse (threshold det_eps) and, when
// jac_noise, Rademacher noise of scale sigma at diffuse vertices.  Attached only.
int or_gradient_literal(const or_scene* s, const or_params* p, const or_run* run, const double* dI,
                        const uint8_t* mask, int jac_noise, uint64_t noise_seed, double sigma, double det_eps,
                        or_grads* out) {
  if (!run->attached) return -1;
  Scene sc{s, p};
  sc.setup();
  int nt = std::max(1, run->n_threads);
  std::vector<Acc> acc(nt);
  const double N = (double)(run->n_norm > 0 ? run->n_norm : run->n_paths);
  const int W = s->W, H = s->H;
  parallel_paths(nt, run->n_paths, [&](int tid, int64_t a, int64_t b) {
    Acc& A = acc[tid];
    A.ga.assign(p->n_albedo, 0.0);
    A.gh.assign(p->n_heights, 0.0);
    Tape tape;
    TP = &tape;
    std::vector<int> node_a(p->n_albedo, -1), node_h(p->n_heights, -1), touch_a, touch_h;
    std::vector<ConnOut<double>> cs;
    std::vector<ConnOut<V>> cv;
    auto flush_h = [&](double w) {  // add w * d(root)/d(heights) of the current tape
      for (int idx : touch_h) A.gh[idx] += w * tape.adj[node_h[idx]];
      for (int idx : touch_h) node_h[idx] = -1;
      touch_h.clear();
    };
    for (int64_t i = a; i < b; ++i) {
      if (mask && !mask[i]) continue;
      const uint64_t n = (uint64_t)(run->path_begin + i);
      Path P = trace(sc, run->seed, n, run->max_depth, run->rr_depth, run->rr_q);
      eval_path<double>(sc, P, Plain{p->albedo}, Plain{p->Le}, Plain{p->heights}, N, cs, &P);
      // (1) naive AD of the frozen path function with the film-position split
      tape.clear();
      touch_a.clear(); touch_h.clear();
      V Lev[3];
      for (int c = 0; c < 3; ++c) Lev[c] = V(p->Le[c], tape.push(-1, 0, -1, 0));
      Leaves la{p->albedo, &node_a, &touch_a}, lh{p->heights, &node_h, &touch_h};
      eval_path<V>(sc, P, la, Lev, lh, N, cv, nullptr, true);
      V loss(0.0);
      for (auto& c : cv) {
        V Lb[3];
        adjoint_read<V>(dI, W, H, c.ux, c.uy, Lb, run->filter);
        loss = loss + c.L[0] * Lb[0] + c.L[1] * Lb[1] + c.L[2] * Lb[2];
      }
      A.loss += loss.v;
      if (loss.i >= 0) {
        tape.backward(loss.i);
        for (int c = 0; c < 3; ++c) A.gL[c] += tape.adj[Lev[c].i];
        for (int idx : touch_a) A.ga[idx] += tape.adj[node_a[idx]];
        for (int idx : touch_h) A.gh[idx] += tape.adj[node_h[idx]];
      }
      for (int idx : touch_a) node_a[idx] = -1;
      for (int idx : touch_h) node_h[idx] = -1;
      touch_h.clear();
      // (2) film-position transport along specular chains (Eq. 18-19)
      const int K = (int)P.v.size();
      if (K < 2 || cs.empty()) continue;
      const Rand4 r0 = rand4(run->seed, n, 0, 0);
      auto prim_of = [&](int j) { return j == 0 ? -1 : P.v[j - 1].prim; };  // vertex j = 1..K, 0 = emitter
      auto coords = [&](int j, double v[2]) {
        if (j == 0) { v[0] = r0.u[0]; v[1] = r0.u[1]; }
        else { v[0] = P.v[j - 1].b1; v[1] = P.v[j - 1].b2; }
      };
      // a_i (position rows of the sensor Jacobian, weighted by dL/du_i) per connection vertex
      std::vector<std::array<double, 4>> arow(K + 1, std::array<double, 4>{0, 0, 0, 0});
      for (auto& c : cs) {
        const int j = c.vi + 1;
        tape.clear();
        V u[2] = {V(c.ux, tape.push(-1, 0, -1, 0)), V(c.uy, tape.push(-1, 0, -1, 0))};
        V Lb[3];
        adjoint_read<V>(dI, W, H, u[0], u[1], Lb, run->filter);
        V term = Lb[0] * V(c.L[0]) + Lb[1] * V(c.L[1]) + Lb[2] * V(c.L[2]);
        double q[2] = {0, 0};
        if (term.i >= 0) { tape.backward(term.i); q[0] = tape.adj[u[0].i]; q[1] = tape.adj[u[1].i]; }
        // du/dv = du/dx [e1 e2] at the vertex's frozen coordinates
        double vv[2];
        coords(j, vv);
        D3 o, e1, e2;
        sc.prim<double>(prim_of(j), p->heights, o, e1, e2);
        for (int d = 0; d < 2; ++d) {
          tape.clear();
          V t0(vv[0], tape.push(-1, 0, -1, 0)), t1(vv[1], tape.push(-1, 0, -1, 0));
          Vec<V> X = lift<V>(o) + lift<V>(e1) * t0 + lift<V>(e2) * t1;
          V ux, uy, zc, dd;
          project<V>(sc, X, ux, uy, zc, dd);
          const V& uo = d == 0 ? ux : uy;
          if (uo.i < 0) continue;
          tape.backward(uo.i);
          arow[j][2] += q[d] * tape.adj[t0.i];
          arow[j][3] += q[d] * tape.adj[t1.i];
        }
      }
      // J_j for j = 1..K-1 and the accumulated products J_{1->j}
      std::vector<std::array<double, 16>> Jacc(K + 1);
      M4 Jp = {{1, 0, 0, 0}, {0, 1, 0, 0}, {0, 0, 1, 0}, {0, 0, 0, 1}};
      std::memcpy(Jacc[1].data(), Jp, sizeof(M4));
      std::vector<bool> spec(K + 1, false);
      // singular by construction once a zero block has entered the product (a diffuse vertex
      // without noise): detected exactly, the determinant guard decides the rest
      std::vector<bool> sing(K + 1, false);
      for (int j = 1; j < K; ++j) {
        sing[j + 1] = sing[j];
        M4 Jj = {{0, 0, 1, 0}, {0, 0, 0, 1}, {0, 0, 0, 0}, {0, 0, 0, 0}};
        const Vtx& vx = P.v[j - 1];
        if (vx.kind == K_SPECULAR) {
          spec[j] = true;
          double vp[2], vj[2];
          coords(j - 1, vp);
          coords(j, vj);
          for (int d = 0; d < 2; ++d) {
            tape.clear();
            V a0(vp[0], tape.push(-1, 0, -1, 0)), a1(vp[1], tape.push(-1, 0, -1, 0));
            V b0(vj[0], tape.push(-1, 0, -1, 0)), b1(vj[1], tape.push(-1, 0, -1, 0));
            const V A2[2] = {a0, a1}, B2[2] = {b0, b1};
            V outv[2];
            spec_next<V>(sc, ConstV{p->heights}, prim_of(j - 1), A2, prim_of(j), B2, vx.refl, prim_of(j + 1), outv);
            if (outv[d].i < 0) continue;
            tape.backward(outv[d].i);
            Jj[2 + d][0] = tape.adj[a0.i]; Jj[2 + d][1] = tape.adj[a1.i];
            Jj[2 + d][2] = tape.adj[b0.i]; Jj[2 + d][3] = tape.adj[b1.i];
          }
        } else if (jac_noise) {
          const double eps = rand4(noise_seed, n, (uint32_t)j, 4).u[0] < 0.5 ? -sigma : sigma;
          Jj[2][0] = eps;
          Jj[3][1] = eps;
        } else {
          sing[j + 1] = true;
        }
        M4 Jn;
        m4_mul(Jj, reinterpret_cast<const double(*)[4]>(Jacc[j].data()), Jn);
        std::memcpy(Jacc[j + 1].data(), Jn, sizeof(M4));
      }
      // A_rem(j) = sum_{i >= j} a_i J_{1->i}; at each specular x_j project A_rem(j+1) with
      // the guarded inverse of J_{1->j+1} and contract with the explicit height dependence
      // of v_{j+1}
      std::array<double, 4> Arem = {0, 0, 0, 0};
      for (int j = K; j >= 1; --j) {
        // Arem currently holds sum_{i > j}; add vertex j's own row
        const double(*Ji)[4] = reinterpret_cast<const double(*)[4]>(Jacc[j].data());
        for (int c = 0; c < 4; ++c)
          for (int k = 0; k < 4; ++k) Arem[c] += arow[j][k] * Ji[k][c];
        // now Arem = A_rem(j); vertex j-1 (if specular) maps p_{j-1} -> p_j
        const int js = j - 1;
        if (js < 1 || !spec[js]) continue;
        M4 inv;
        if (sing[j] || !m4_inv(Ji, inv, det_eps)) continue;
        double aloc[4] = {0, 0, 0, 0};
        for (int c = 0; c < 4; ++c)
          for (int k = 0; k < 4; ++k) aloc[c] += Arem[k] * inv[k][c];
        if (aloc[2] == 0.0 && aloc[3] == 0.0) continue;
        double vp[2], vj[2];
        coords(js - 1, vp);
        coords(js, vj);
        tape.clear();
        touch_h.clear();
        const V A2[2] = {V(vp[0]), V(vp[1])}, B2[2] = {V(vj[0]), V(vj[1])};
        V outv[2];
        spec_next<V>(sc, lh, prim_of(js - 1), A2, prim_of(js), B2, P.v[js - 1].refl, prim_of(js + 1), outv);
        V w = outv[0] * V(aloc[2]) + outv[1] * V(aloc[3]);
        if (w.i >= 0) {
          tape.backward(w.i);
          flush_h(1.0);
        } else {
          for (int idx : touch_h) node_h[idx] = -1;
          touch_h.clear();
        }
      }
    }
    TP = nullptr;
  });
  if (out->d_albedo)
    for (int j = 0; j < p->n_albedo; ++j) { double v = 0; for (int t = 0; t < nt; ++t) if (acc[t].ga.size()) v += acc[t].ga[j]; out->d_albedo[j] = v; }
  if (out->d_heights)
    for (int j = 0; j < p->n_heights; ++j) { double v = 0; for (int t = 0; t < nt; ++t) if (acc[t].gh.size()) v += acc[t].gh[j]; out->d_heights[j] = v; }
  if (out->d_Le) for (int c = 0; c < 3; ++c) { double v = 0; for (int t = 0; t < nt; ++t) v += acc[t].gL[c]; out->d_Le[c] = v; }
  if (out->loss) { double v = 0; for (int t = 0; t < nt; ++t) v += acc[t].loss; out->loss[0] = v; }
  return 0;
}

// Camera-side path tracer with next-event estimation to the area emitter (radiance
// transport; used only to pin the light tracer by reciprocity: Eq. 1 measured from the
// sensor side, Sec. 3.1).  Pixel p estimates
// integral of tent_p(u) L(camera ray through u) du with u sampled from the tent itself;
// camera paths with 1..D surface vertices are counted through NEE at each diffuse vertex
// (matching light paths x0..xi with i <= D); emitter hits are black.  Diffuse scenes only.
int or_render_pt(const or_scene* s, const or_params* p, uint64_t seed, int spp, int max_depth, int n_threads,
                 double* image) {
  Scene sc{s, p};
  sc.setup();
  const int W = s->W, H = s->H;
  D3 lo, le1, le2;
  sc.prim<double>(s->emitter_quad, p->heights, lo, le1, le2);
  D3 nL = normalize(cross(le1, le2));
  double A_L = norm(cross(le1, le2));
  auto tent_sample = [](double u) { return u < 0.5 ? std::sqrt(2 * u) - 1 : 1 - std::sqrt(2 - 2 * u); };
  parallel_paths(n_threads, (int64_t)W * H, [&](int, int64_t a, int64_t b) {
    for (int64_t pix = a; pix < b; ++pix) {
      int px = (int)(pix % W), py = (int)(pix / W);
      double sum[3] = {0, 0, 0};
      for (int smp = 0; smp < spp; ++smp) {
        uint64_t pid = (uint64_t)pix * (uint64_t)spp + (uint64_t)smp;
        Rand4 r0 = rand4(seed, pid, 0, 1);
        double ux = px + 0.5 + tent_sample(r0.u[0]), uy = py + 0.5 + tent_sample(r0.u[1]);
        if (!(ux >= 0 && ux < W && uy >= 0 && uy < H)) continue;
        double pxn = (2 * ux / W - 1) * sc.tanx, pyn = (1 - 2 * uy / H) * sc.tany;
        D3 dir = normalize(sc.cf + sc.cr * pxn + sc.cu * pyn);
        D3 org = sc.cpos;
        int skip = -1;
        double thr[3] = {1, 1, 1};
        for (int m = 1; m <= max_depth; ++m) {
          int prim;
          double tt, su, sv;
          if (!closest(sc, org, dir, skip, prim, tt, su, sv)) break;
          int mt = sc.mtype(prim);
          if (mt != 0) break;  // emitter (black) ; dielectrics unsupported here
          D3 o, e1, e2;
          sc.prim<double>(prim, p->heights, o, e1, e2);
          D3 x = o + e1 * su + e2 * sv;
          D3 nrm = normalize(cross(e1, e2));
          D3 ns = dot(nrm, dir) < 0 ? nrm : nrm * -1.0;
          double rho[3];
          tex_lookup<double>(sc, sc.mat(prim), Plain{p->albedo}, su, sv, rho);
          Rand4 r = rand4(seed, pid, (uint32_t)m, 1);
          D3 y = lo + le1 * r.u[0] + le2 * r.u[1];
          D3 wl = y - x;
          double dist = norm(wl);
          D3 wn = wl * (1.0 / dist);
          double cx = dot(ns, wn), cl = -dot(nL, wn);
          if (cx > 0 && cl > 0 && !occluded(sc, x, wn, dist, prim)) {
            double gterm = cx * cl / (dist * dist) * A_L / PI;
            for (int c = 0; c < 3; ++c) sum[c] += thr[c] * rho[c] * p->Le[c] * gterm;
          }
          D3 ta, tb;
          onb(ns, ta, tb);
          double r1 = std::sqrt(r.u[2]), p1 = 2 * PI * r.u[3];
          dir = ta * (r1 * std::cos(p1)) + tb * (r1 * std::sin(p1)) + ns * std::sqrt(std::max(0.0, 1 - r.u[2]));
          for (int c = 0; c < 3; ++c) thr[c] *= rho[c];
          org = x;
          skip = prim;
        }
      }
      for (int c = 0; c < 3; ++c) image[pix * 3 + c] = sum[c] / spp;
    }
  });
  return 0;
}

}  // extern "C"

// =============================================================== learned reservoir target
// FP64 reference of the 16 -> 64 -> 64 -> 1 ReLU network (parameter block layout as the
// library's: W1[16][64] b1[64] W2[64][64] b2[64] W3[64] b3 | mean[16] 1/std[16] | target
// scale, target mean).  With `round` set it applies the same BFloat16 roundings as the
// tensor-core path (standardized inputs, weights W1 W2 W3, hidden activations after ReLU);
// the backward treats those roundings as identity (straight-through).
namespace {
double bf16_round(double x) {
  float f = (float)x;
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);  // round to nearest even on the upper 16 bits
  u &= 0xFFFF0000u;
  std::memcpy(&f, &u, 4);
  return (double)f;
}
struct MlpRef {
  const double* P;
  bool round;
  double W1(int k, int o) const { double w = P[k * 64 + o]; return round ? bf16_round(w) : w; }
  double W2(int k, int o) const { double w = P[1088 + k * 64 + o]; return round ? bf16_round(w) : w; }
  double W3(int k) const { double w = P[5248 + k]; return round ? bf16_round(w) : w; }
  void forward(const double* f, double x[16], double z1[64], double h1[64], double z2[64], double h2[64], double& y) const {
    for (int i = 0; i < 16; ++i) {
      x[i] = (double)(float)(((float)f[i] - (float)P[5313 + i]) * (float)P[5329 + i]);
      if (round) x[i] = bf16_round(x[i]);
    }
    for (int o = 0; o < 64; ++o) {
      double a = P[1024 + o];
      for (int k = 0; k < 16; ++k) a += x[k] * W1(k, o);
      z1[o] = a;
      h1[o] = a > 0 ? a : 0.0;
      if (round) h1[o] = bf16_round(h1[o]);
    }
    for (int o = 0; o < 64; ++o) {
      double a = P[5184 + o];
      for (int k = 0; k < 64; ++k) a += h1[k] * W2(k, o);
      z2[o] = a;
      h2[o] = a > 0 ? a : 0.0;
      if (round) h2[o] = bf16_round(h2[o]);
    }
    y = P[5312];
    for (int k = 0; k < 64; ++k) y += h2[k] * W3(k);
  }
};
}  // namespace

extern "C" {
// The learned reservoir target's network (not in the paper: 16 -> 64 -> 64 -> 1, ReLU),
// optionally with the BF16 roundings of the GPU path; outputs in standardised units.
void or_mlp_forward(const double* P, const double* X, int64_t n, int round, double* out) {
  MlpRef M{P, round != 0};
  for (int64_t s = 0; s < n; ++s) {
    double x[16], z1[64], h1[64], z2[64], h2[64], y;
    M.forward(X + 16 * s, x, z1, h1, z2, h2, y);
    out[s] = y;
  }
}

// Gradient of L = (1/n) sum_s (y_s - t_s)^2 with t_s = (T_s - target mean) / target scale,
// by hand-written reverse mode (chain rule through the three layers).
double or_mlp_grad(const double* P, const double* X, const double* T, int64_t n, int round, double* grad) {
  MlpRef M{P, round != 0};
  for (int i = 0; i < 5313; ++i) grad[i] = 0.0;
  double loss = 0.0;
  for (int64_t s = 0; s < n; ++s) {
    double x[16], z1[64], h1[64], z2[64], h2[64], y;
    M.forward(X + 16 * s, x, z1, h1, z2, h2, y);
    const double t = (T[s] - P[5346]) / P[5345];
    const double e = y - t;
    loss += e * e / (double)n;
    const double dy = 2.0 * e / (double)n;
    grad[5312] += dy;
    double dz2[64], dh1[64];
    for (int k = 0; k < 64; ++k) {
      grad[5248 + k] += dy * h2[k];
      dz2[k] = z2[k] > 0 ? dy * M.W3(k) : 0.0;
      grad[5184 + k] += dz2[k];
    }
    for (int i = 0; i < 64; ++i) {
      double a = 0.0;
      for (int j = 0; j < 64; ++j) {
        grad[1088 + i * 64 + j] += h1[i] * dz2[j];
        a += dz2[j] * M.W2(i, j);
      }
      dh1[i] = a;
    }
    for (int i = 0; i < 64; ++i) {
      const double dz1 = z1[i] > 0 ? dh1[i] : 0.0;
      grad[1024 + i] += dz1;
      for (int k = 0; k < 16; ++k) grad[k * 64 + i] += x[k] * dz1;
    }
  }
  return loss;
}
}  // extern "C"

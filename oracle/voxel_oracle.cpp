// FP64 reference ("oracle") for the voxel lattice simulator of Hiller & Lipson,
// "Dynamic Simulation of Soft Heterogeneous Objects" (arXiv 1212.2845).
//
// TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the
// CPU-baseline leg of the benchmark load this library.  It shares no code,
// header, table or constant generator with the CUDA path.
//
// It is deliberately plain and slow: every step follows the paper in its own
// order (Section 2.1: compute all bond forces, then update every voxel
// synchronously), with no blocking, fusion or reordering.  All arithmetic is
// templated on the scalar type R so that the same code runs in double and in
// a forward-mode dual number (exact directional derivatives for checking
// gradients).
//
// Readings of the paper where it is silent, garbled or self-contradictory are
// marked "READING" and listed in the design notes of the repository.
//
// Parity status per function (what pins it; see tests/test_oracle_*.py):
//   composite material (Sec 2.1.1, Eqs E_c, G_c)     pinned: single-bond stiffness
//   beam constants (Sec 2.1.2, a1..b3)                 pinned: cantilever closed form
//   bond force (Sec 2.1.2 reduced equations)           pinned: Jacobian == printed [K]
//   integration (Sec 2.1.3)                            pinned: free flight, conservation
//   stable timestep (Sec 2.1.4)                        pinned: closed form (test retypes
//                                                      nothing: checks stability + value)
//   bond damping (Sec 2.1.5)                           pinned: rigid motion undamped
//   gravity/floor/friction (Sec 2.2.1)                 pinned: friction threshold/decel.
//   collision candidates (Sec 2.2.2)                   pinned: brute-force sets; the
//                                                      x-sorted sweep equals brute force
//   voxel-voxel contact force law (paper silent)       pinned: one-step force, rest
//                                                      overlap m g / k_c, restitution
//                                                      and contact time of a head-on
//                                                      damped collision
//   volumetric actuation (Sec 2.3)                     pinned: free expansion
//   several temperature signals (Sec 2.3)              pinned: two-material rest length,
//                                                      solo runs of one-material bodies
//   bodies in one world (Sec 2.2.2)                    pinned: antisymmetric cross-body
//                                                      pairs (momentum), bounce
//   collision schemes (all/surface, every/horizon)     pinned: identical trajectories
//   assembled stiffness (modal check)                  pinned: beam-theory frequencies
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

namespace orc {

// ---------------------------------------------------------------------------
// Scalar types: double and a first-order forward-mode dual number.
// ---------------------------------------------------------------------------
struct Dual {
  double v, d;
  Dual(double a = 0.0, double b = 0.0) : v(a), d(b) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
  return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
inline Dual& operator*=(Dual& a, Dual b) { a = a * b; return a; }
inline bool operator<(Dual a, Dual b) { return a.v < b.v; }
inline bool operator>(Dual a, Dual b) { return a.v > b.v; }
inline bool operator<=(Dual a, Dual b) { return a.v <= b.v; }
inline bool operator>=(Dual a, Dual b) { return a.v >= b.v; }
inline Dual sqrt(Dual a) { double s = std::sqrt(a.v); return Dual(s, s > 0 ? a.d / (2 * s) : 0.0); }
inline Dual sin(Dual a) { return Dual(std::sin(a.v), a.d * std::cos(a.v)); }
inline Dual cos(Dual a) { return Dual(std::cos(a.v), -a.d * std::sin(a.v)); }
inline Dual exp(Dual a) { double e = std::exp(a.v); return Dual(e, a.d * e); }
inline Dual atan2(Dual y, Dual x) {
  double r2 = x.v * x.v + y.v * y.v;
  return Dual(std::atan2(y.v, x.v), (x.v * y.d - y.v * x.d) / r2);
}
inline double val(double a) { return a; }
inline double val(const Dual& a) { return a.v; }
using std::sqrt; using std::sin; using std::cos; using std::exp; using std::atan2;

// ---------------------------------------------------------------------------
// Small vector / quaternion algebra (generic in R)
// ---------------------------------------------------------------------------
template <class R> struct V3 {
  R x, y, z;
  V3() : x(0.0), y(0.0), z(0.0) {}
  V3(R a, R b, R c) : x(a), y(b), z(c) {}
  R& operator[](int i) { return i == 0 ? x : (i == 1 ? y : z); }
  const R& operator[](int i) const { return i == 0 ? x : (i == 1 ? y : z); }
};
template <class R> V3<R> operator+(const V3<R>& a, const V3<R>& b) { return V3<R>(a.x + b.x, a.y + b.y, a.z + b.z); }
template <class R> V3<R> operator-(const V3<R>& a, const V3<R>& b) { return V3<R>(a.x - b.x, a.y - b.y, a.z - b.z); }
template <class R> V3<R> operator-(const V3<R>& a) { return V3<R>(-a.x, -a.y, -a.z); }
template <class R> V3<R> operator*(const V3<R>& a, R s) { return V3<R>(a.x * s, a.y * s, a.z * s); }
template <class R> V3<R> operator*(R s, const V3<R>& a) { return V3<R>(a.x * s, a.y * s, a.z * s); }
template <class R> V3<R>& operator+=(V3<R>& a, const V3<R>& b) { a = a + b; return a; }
template <class R> V3<R>& operator-=(V3<R>& a, const V3<R>& b) { a = a - b; return a; }
template <class R> R dot(const V3<R>& a, const V3<R>& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class R> V3<R> cross(const V3<R>& a, const V3<R>& b) {
  return V3<R>(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// Unit quaternion q = (w, x, y, z); R(q) maps a voxel's body frame to the world.
template <class R> struct Q4 {
  R w, x, y, z;
  Q4() : w(1.0), x(0.0), y(0.0), z(0.0) {}
  Q4(R a, R b, R c, R d) : w(a), x(b), y(c), z(d) {}
};
template <class R> Q4<R> qmul(const Q4<R>& a, const Q4<R>& b) {
  return Q4<R>(a.w * b.w - a.x * b.x - a.y * b.y - a.z * b.z,
               a.w * b.x + a.x * b.w + a.y * b.z - a.z * b.y,
               a.w * b.y - a.x * b.z + a.y * b.w + a.z * b.x,
               a.w * b.z + a.x * b.y - a.y * b.x + a.z * b.w);
}
template <class R> Q4<R> qconj(const Q4<R>& a) { return Q4<R>(a.w, -a.x, -a.y, -a.z); }
// v' = q (0,v) q*
template <class R> V3<R> qrot(const Q4<R>& q, const V3<R>& v) {
  Q4<R> p(R(0.0), v.x, v.y, v.z);
  Q4<R> r = qmul(qmul(q, p), qconj(q));
  return V3<R>(r.x, r.y, r.z);
}
template <class R> V3<R> qrot_inv(const Q4<R>& q, const V3<R>& v) { return qrot(qconj(q), v); }
template <class R> Q4<R> qnormalize(const Q4<R>& q) {
  R n = sqrt(q.w * q.w + q.x * q.x + q.y * q.y + q.z * q.z);
  return Q4<R>(q.w / n, q.x / n, q.y / n, q.z / n);
}
// Rotation vector (axis * angle) of a unit quaternion, shortest arc.
template <class R> V3<R> qlog_vec(Q4<R> q) {
  if (val(q.w) < 0.0) q = Q4<R>(-q.w, -q.x, -q.y, -q.z);
  R s2 = q.x * q.x + q.y * q.y + q.z * q.z;
  R f;  // angle / |v| = 2 atan2(s, w) / s
  if (val(s2) < 1e-16) {
    // series of 2 atan(t)/t at t = s/w -> 2/w (1 - t^2/3); exact to O(t^4)
    R t2 = s2 / (q.w * q.w);
    f = R(2.0) / q.w * (R(1.0) - t2 / R(3.0));
  } else {
    R s = sqrt(s2);
    f = R(2.0) * atan2(s, q.w) / s;
  }
  return V3<R>(q.x * f, q.y * f, q.z * f);
}
// Quaternion of the rotation by vector w (angle |w| about w/|w|).
template <class R> Q4<R> qexp_vec(const V3<R>& w) {
  R a2 = dot(w, w);
  R half2 = a2 / R(4.0);  // (|w|/2)^2
  R c, k;                 // cos(|w|/2), sin(|w|/2)/|w|
  if (val(half2) < 1e-16) {
    c = R(1.0) - half2 / R(2.0);
    k = R(0.5) * (R(1.0) - half2 / R(6.0));
  } else {
    R a = sqrt(a2);
    c = cos(a / R(2.0));
    k = sin(a / R(2.0)) / a;
  }
  return Q4<R>(c, w.x * k, w.y * k, w.z * k);
}

// Cyclic permutation Pi_a taking the bond axis a to local x (a proper rotation):
// local[i] = v[(i + a) % 3].  READING: the paper only says elements are rotated
// "into the positive X direction" (Sec 2.1.2); a cyclic permutation is the
// rotation that does so without a reflection.
template <class R> V3<R> to_axis(const V3<R>& v, int a) { return V3<R>(v[a % 3], v[(a + 1) % 3], v[(a + 2) % 3]); }
template <class R> V3<R> from_axis(const V3<R>& u, int a) {
  V3<R> v;
  v[a % 3] = u.x; v[(a + 1) % 3] = u.y; v[(a + 2) % 3] = u.z;
  return v;
}

// ---------------------------------------------------------------------------
// Topology: occupied sites, bonds, surface voxels (integer, shared by all R)
// ---------------------------------------------------------------------------
struct Topo {
  int n_bodies = 0;
  std::vector<std::array<int, 3>> dims;
  double l = 0.0;
  int N = 0;
  std::vector<int> body, vi, vj, vk, mat;  // per voxel, canonical order; mat is 0-based
  std::vector<std::array<int, 6>> nbr;     // -x,+x,-y,+y,-z,+z neighbour (same body) or -1
  struct Bond { int v1, v2, axis; };
  std::vector<Bond> bonds;                 // v1 on the negative side of the axis
  std::vector<std::array<int, 6>> slot_bond;  // bond id per neighbour slot or -1
  std::vector<uint8_t> surface;            // 1 if fewer than 6 occupied face neighbours
  std::vector<int> body_first;             // first voxel of each body (+ sentinel)
};

static void build_topology(Topo& T, int n_bodies, const int32_t* dims, const uint8_t* grid, double l) {
  T.n_bodies = n_bodies;
  T.l = l;
  T.dims.resize(n_bodies);
  std::vector<std::vector<int>> site_to_voxel(n_bodies);
  size_t off = 0;
  T.body_first.clear();
  for (int b = 0; b < n_bodies; ++b) {
    int nx = dims[3 * b], ny = dims[3 * b + 1], nz = dims[3 * b + 2];
    T.dims[b] = {nx, ny, nz};
    site_to_voxel[b].assign((size_t)nx * ny * nz, -1);
    T.body_first.push_back((int)T.body.size());
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
          size_t s = (size_t)i + (size_t)nx * ((size_t)j + (size_t)ny * k);
          uint8_t m = grid[off + s];
          if (m == 0) continue;
          site_to_voxel[b][s] = (int)T.body.size();
          T.body.push_back(b); T.vi.push_back(i); T.vj.push_back(j); T.vk.push_back(k);
          T.mat.push_back(m - 1);
        }
    off += (size_t)nx * ny * nz;
  }
  T.body_first.push_back((int)T.body.size());
  T.N = (int)T.body.size();
  T.nbr.assign(T.N, {-1, -1, -1, -1, -1, -1});
  T.slot_bond.assign(T.N, {-1, -1, -1, -1, -1, -1});
  T.surface.assign(T.N, 0);
  T.bonds.clear();
  for (int v = 0; v < T.N; ++v) {
    int b = T.body[v];
    auto d = T.dims[b];
    int c[3] = {T.vi[v], T.vj[v], T.vk[v]};
    int occupied = 0;
    for (int a = 0; a < 3; ++a)
      for (int s = 0; s < 2; ++s) {
        int cc[3] = {c[0], c[1], c[2]};
        cc[a] += (s == 0 ? -1 : 1);
        int u = -1;
        if (cc[a] >= 0 && cc[a] < d[a]) u = site_to_voxel[b][(size_t)cc[0] + (size_t)d[0] * ((size_t)cc[1] + (size_t)d[1] * cc[2])];
        T.nbr[v][2 * a + s] = u;
        if (u >= 0) ++occupied;
      }
    T.surface[v] = occupied < 6 ? 1 : 0;
  }
  for (int v = 0; v < T.N; ++v)
    for (int a = 0; a < 3; ++a) {
      int u = T.nbr[v][2 * a + 1];
      if (u < 0) continue;
      int id = (int)T.bonds.size();
      T.bonds.push_back({v, u, a});
      T.slot_bond[v][2 * a + 1] = id;
      T.slot_bond[u][2 * a] = id;
    }
}

// Collision quantisation (see the design notes): positions are offsets o from
// the voxel's lattice anchor (its rest centre); a coordinate becomes the
// integer anchor*Q + rint(o * 2^K), where 2^K <= 65536/l < 2^(K+1) and
// Q = rint(l * 2^K).  Scaling by 2^K is exact in binary floating point.
static void quant_params(double l, int* K, int64_t* Q) {
  int e;
  std::frexp(65536.0 / l, &e);   // 65536/l = m 2^e, m in [0.5, 1)
  *K = e - 1;
  *Q = (int64_t)std::nearbyint(std::ldexp(l, *K));
}

// ---------------------------------------------------------------------------
// Simulator state and parameters
// ---------------------------------------------------------------------------
struct Params {
  double zeta_bond = 1.0, zeta_ground = 0.0, zeta_collision = 1.0;
  double gravity_z = 0.0;
  int floor_on = 0, collide_on = 0;
  // collision scheme (the paper's comparison): candidates among all voxels
  // instead of surface voxels; rebuild every step instead of on the horizon
  int cand_all = 0, cand_every = 0;
  // test every pair of searched voxels instead of the sorted sweep (same set)
  int brute_search = 0;
  double act_A = 0.0, act_T0 = 0.0;
  long act_P = 0;
  // several temperature signals (Sec 2.3): per material amplitude, offset and
  // phase shift on the common period; empty = the single global signal
  std::vector<double> mat_A, mat_T0, mat_ph;
  double dt_factor = 0.9;
};

template <class R> struct Sim {
  Topo T;
  Params prm;
  std::vector<double> pal;     // n_mat x 6: E, nu, rho, cte, mu_s, mu_k
  int n_mat = 0;
  std::vector<V3<double>> origin;  // per body
  // per voxel
  std::vector<R> E, G, phase;
  std::vector<double> rho, cte, mus, muk, mass, inertia;
  std::vector<uint8_t> fixed;
  std::vector<V3<double>> Fext;
  // state: position D, orientation q, linear momentum P, angular momentum phi
  // (Sec 2.1.3 notation), static-friction flag
  std::vector<V3<R>> D, P, phi;
  std::vector<Q4<R>> q;
  std::vector<uint8_t> stat;
  std::vector<double> dt;      // per body, frozen (never differentiated)
  long n = 0;                  // step counter
  // collisions
  std::vector<double> acc;     // per body max-motion accumulator (Sec 2.2.2)
  std::vector<std::vector<int>> partners;  // per voxel, ascending
  long n_rebuilds = 0;
  int qK = 0; int64_t qQ = 0;
  // signature of the run's discrete decisions (floor contact and its
  // stick/slip branch, voxel-voxel contacts): two runs that take the same
  // branches everywhere have the same signature (test aid for finite
  // differences, which are only meaningful when no decision flips inside +-h)
  uint64_t events = 1469598103934665603ull;
  // per-step scratch
  struct BondOut { V3<R> F1, M1, F2, M2; };
  std::vector<BondOut> bo;

  V3<double> anchor(int v) const {
    const V3<double>& o = origin[T.body[v]];
    return V3<double>(o.x + (T.vi[v] + 0.5) * T.l, o.y + (T.vj[v] + 0.5) * T.l, o.z + (T.vk[v] + 0.5) * T.l);
  }
};

// Composite properties of a bond (Sec 2.1.1) and beam constants (Sec 2.1.2).
template <class R> struct BeamK { R a1, a2, b1, b2, b3; };
template <class R> static BeamK<R> beam_constants(const Sim<R>& S, int v1, int v2) {
  R E1 = S.E[v1], E2 = S.E[v2], G1 = S.G[v1], G2 = S.G[v2];
  R Ec = R(2.0) * E1 * E2 / (E1 + E2);
  R Gc = R(2.0) * G1 * G2 / (G1 + G2);
  double l = S.T.l;
  double A = l * l, I = l * l * l * l / 12.0, J = l * l * l * l / 6.0;
  BeamK<R> k;
  k.a1 = Ec * R(A / l);
  k.a2 = Gc * R(J / l);
  k.b1 = R(12.0) * Ec * R(I / (l * l * l));
  k.b2 = R(6.0) * Ec * R(I / (l * l));
  k.b3 = R(2.0) * Ec * R(I / l);
  return k;
}

template <class R> static void set_materials(Sim<R>& S, const double* logE) {
  const Topo& T = S.T;
  int N = T.N;
  S.E.resize(N); S.G.resize(N);
  S.rho.resize(N); S.cte.resize(N); S.mus.resize(N); S.muk.resize(N);
  S.mass.resize(N); S.inertia.resize(N);
  double l = T.l;
  for (int v = 0; v < N; ++v) {
    const double* m = &S.pal[6 * T.mat[v]];
    R Ev = logE ? exp(R(logE[v])) : R(m[0]);
    S.E[v] = Ev;
    S.G[v] = Ev / R(2.0 * (1.0 + m[1]));
    S.rho[v] = m[2]; S.cte[v] = m[3]; S.mus[v] = m[4]; S.muk[v] = m[5];
    S.mass[v] = m[2] * l * l * l;
    S.inertia[v] = S.mass[v] * l * l / 6.0;  // READING: solid cube, m l^2 / 6
  }
}

// Stable timestep (Sec 2.1.4): dt = f / (2 pi omega_max), omega = sqrt(k_b / m_min)
// maximised over the bonds of each body.  READING: a voxel's own floor/contact
// spring k_v = E_v l on its own mass counts as a bond for this maximum.
template <class R> static void compute_dt(Sim<R>& S) {
  const Topo& T = S.T;
  std::vector<double> wmax(T.n_bodies, 0.0);
  for (const auto& bd : T.bonds) {
    BeamK<R> k = beam_constants(S, bd.v1, bd.v2);
    double m = std::min(S.mass[bd.v1], S.mass[bd.v2]);
    double w = std::sqrt(val(k.a1) / m);
    int b = T.body[bd.v1];
    wmax[b] = std::max(wmax[b], w);
  }
  for (int v = 0; v < T.N; ++v) {
    double w = std::sqrt(val(S.E[v]) * T.l / S.mass[v]);
    wmax[T.body[v]] = std::max(wmax[T.body[v]], w);
  }
  S.dt.assign(T.n_bodies, 0.0);
  for (int b = 0; b < T.n_bodies; ++b)
    S.dt[b] = wmax[b] > 0 ? S.prm.dt_factor / (2.0 * M_PI * wmax[b]) : 0.0;
  if (S.prm.collide_on == 2) {  // one world, one clock: the smallest timestep
    double dmin = 0.0;
    for (int b = 0; b < T.n_bodies; ++b)
      if (S.dt[b] > 0 && (dmin == 0.0 || S.dt[b] < dmin)) dmin = S.dt[b];
    for (int b = 0; b < T.n_bodies; ++b) S.dt[b] = dmin;
  }
}

// Temperature offset of a voxel at step n (Sec 2.3): T_c - T_r.
// Each material follows its own signal when one is set, else the global one.
static void signal_of(const Params& p, int m, double* A, double* T0, double* ph) {
  *A = p.mat_A.empty() ? p.act_A : p.mat_A[m];
  *T0 = p.mat_T0.empty() ? p.act_T0 : p.mat_T0[m];
  *ph = p.mat_ph.empty() ? 0.0 : p.mat_ph[m];
}

template <class R> static R delta_T(const Sim<R>& S, int v) {
  const Params& p = S.prm;
  double A, T0, ph;
  signal_of(p, S.T.mat[v], &A, &T0, &ph);
  if (p.act_P > 0)
    return R(T0) + R(A) * sin(R(2.0 * M_PI * (double)S.n / (double)p.act_P) + S.phase[v] + R(ph));
  return R(T0);
}

// Force and moment of one bond on its two voxels (Sec 2.1.2, 2.1.5, 2.3).
template <class R> static void bond_force(const Sim<R>& S, int id, const std::vector<R>& dT,
                                          typename Sim<R>::BondOut& out) {
  const auto& bd = S.T.bonds[id];
  int v1 = bd.v1, v2 = bd.v2, a = bd.axis;
  BeamK<R> k = beam_constants(S, v1, v2);
  // Volumetric actuation: rest length scaled by 1 + (a1 dT1 + a2 dT2)/2 (Eq. of Sec 2.3;
  // READING: per-voxel temperatures enter as the mean of the two strains).
  R eps = R(0.5) * (R(S.cte[v1]) * dT[v1] + R(S.cte[v2]) * dT[v2]);
  R L0 = R(S.T.l) * (R(1.0) + eps);
  // Translate and rotate so voxel 1 sits at zero position and zero angle (Sec 2.1.2).
  const Q4<R>& q1 = S.q[v1];
  V3<R> p = to_axis(qrot_inv(q1, S.D[v2] - S.D[v1]), a);
  V3<R> th = to_axis(qlog_vec(qmul(qconj(q1), S.q[v2])), a);
  R X = p.x - L0, Y = p.y, Z = p.z;
  // Rows of [K] u with the first voxel's DOFs zero (reduced equations).
  // READING: the printed F_z1 = -b1 Z2 + b2 theta_y2 contradicts row 3 of [K]
  // (and F_z2 = -F_z1); the matrix gives -b1 Z2 - b2 theta_y2, used here.
  V3<R> Fk1(-k.a1 * X, -k.b1 * Y + k.b2 * th.z, -k.b1 * Z - k.b2 * th.y);
  V3<R> Mk1(-k.a2 * th.x, k.b2 * Z + k.b3 * th.y, -k.b2 * Y + k.b3 * th.z);
  V3<R> Fk2 = -Fk1;
  V3<R> Mk2(k.a2 * th.x, k.b2 * Z + R(2.0) * k.b3 * th.y, -k.b2 * Y + R(2.0) * k.b3 * th.z);
  // READING: [K]u are the nodal forces that hold the deformed shape; the
  // bond pulls its voxels back with the opposite sign.  Back to world frame.
  out.F1 = qrot(q1, from_axis(-Fk1, a));
  out.M1 = qrot(q1, from_axis(-Mk1, a));
  out.F2 = qrot(q1, from_axis(-Fk2, a));
  out.M2 = qrot(q1, from_axis(-Mk2, a));
  // Local bond damping (Sec 2.1.5): velocity of voxel 2 relative to the
  // bond's rigid motion; READING: m and I are the smaller of the two voxels',
  // k is a1 for translation and b3 for rotation (sqrt(b3/I) equals
  // sqrt(a1/m), so both dampers have the same rate; with the bending diagonal
  // 2 b3 a solid lattice diverges at zeta = 1 under the paper's timestep).
  double zb = S.prm.zeta_bond;
  if (zb != 0.0) {
    V3<R> v1v = S.P[v1] * R(1.0 / S.mass[v1]), v2v = S.P[v2] * R(1.0 / S.mass[v2]);
    V3<R> w1 = S.phi[v1] * R(1.0 / S.inertia[v1]), w2 = S.phi[v2] * R(1.0 / S.inertia[v2]);
    V3<R> Va = (v1v + v2v) * R(0.5), wa = (w1 + w2) * R(0.5), Da = (S.D[v1] + S.D[v2]) * R(0.5);
    V3<R> V21 = (v2v - Va) + cross(S.D[v2] - Da, wa);
    double mmin = std::min(S.mass[v1], S.mass[v2]);
    double Imin = std::min(S.inertia[v1], S.inertia[v2]);
    R c = R(2.0 * zb) * sqrt(R(mmin) * k.a1);
    R cr = R(2.0 * zb) * sqrt(R(Imin) * k.b3);
    out.F2 -= V21 * c;
    out.F1 += V21 * c;
    out.M2 -= (w2 - wa) * cr;
    out.M1 -= (w1 - wa) * cr;
  }
}

// Collision candidates (Sec 2.2.2): surface voxels i<j, quantised centre
// distance < 2 voxels; two voxels of one body must also be more than 3 apart
// in lattice Manhattan distance.  Voxels of different bodies pair only in the
// shared-world mode (collide_on == 2: all bodies in one world), where they
// are never excluded.
template <class R> static bool cand_pred(const Sim<R>& S, int i, int j, const std::vector<std::array<int64_t, 3>>& xq) {
  const Topo& T = S.T;
  if (T.body[i] != T.body[j]) {
    if (S.prm.collide_on != 2) return false;
  } else {
    int man = std::abs(T.vi[i] - T.vi[j]) + std::abs(T.vj[i] - T.vj[j]) + std::abs(T.vk[i] - T.vk[j]);
    if (man <= 3) return false;
  }
  int64_t dx = xq[i][0] - xq[j][0], dy = xq[i][1] - xq[j][1], dz = xq[i][2] - xq[j][2];
  int64_t two = 2 * S.qQ;
  return dx * dx + dy * dy + dz * dz < two * two;
}

// Quantised centre: lattice index * Q + rint(offset * 2^K), plus in the
// shared-world mode the body origin rint(origin * 2^K), so that all bodies
// share one integer frame.
template <class R> static std::vector<std::array<int64_t, 3>> quantise_positions(const Sim<R>& S) {
  const Topo& T = S.T;
  std::vector<std::array<int64_t, 3>> xq(T.N);
  for (int v = 0; v < T.N; ++v) {
    V3<double> an = S.anchor(v);
    int c[3] = {T.vi[v], T.vj[v], T.vk[v]};
    const V3<double>& org = S.origin[T.body[v]];
    for (int a = 0; a < 3; ++a) {
      double o = val(S.D[v][a]) - an[a];
      int64_t qo = S.prm.collide_on == 2 ? (int64_t)std::nearbyint(std::ldexp(org[a], S.qK)) : 0;
      xq[v][a] = qo + (int64_t)c[a] * S.qQ + (int64_t)std::nearbyint(std::ldexp(o, S.qK));
    }
  }
  return xq;
}

// The candidate pairs (i < j) among the searched voxels `list` (Sec 2.2.2)
// for the quantised centres xq, in no particular order.  Brute force tests
// every pair.  The default search visits the voxels in order of their
// quantised x coordinate and tests, for each, only the voxels after it whose
// x differs by less than 2 Q: a pair with |dx| >= 2 Q has dx^2 >= (2 Q)^2 and
// fails the strict distance test, so both searches find the same set
// (checked against each other by the tests).
template <class R> static std::vector<std::pair<int, int>> find_pairs(const Sim<R>& S, const std::vector<int>& list,
                                                                     const std::vector<std::array<int64_t, 3>>& xq) {
  std::vector<std::pair<int, int>> out;
  const size_t n = list.size();
  auto test = [&](int i, int j) {
    if (cand_pred(S, i, j, xq)) out.push_back(i < j ? std::make_pair(i, j) : std::make_pair(j, i));
  };
  if (S.prm.brute_search) {
    for (size_t a = 0; a < n; ++a)
      for (size_t b = a + 1; b < n; ++b) test(list[a], list[b]);
    return out;
  }
  std::vector<int> ord(list);
  std::sort(ord.begin(), ord.end(), [&](int u, int v) { return xq[u][0] < xq[v][0] || (xq[u][0] == xq[v][0] && u < v); });
  const int64_t two = 2 * S.qQ;
  for (size_t a = 0; a < n; ++a)
    for (size_t b = a + 1; b < n && xq[ord[b]][0] - xq[ord[a]][0] < two; ++b) test(ord[a], ord[b]);
  return out;
}

// The pairs of `list` written into the partner lists of its voxels (cleared
// first, sorted ascending).
template <class R> static void search_pairs(Sim<R>& S, const std::vector<int>& list,
                                            const std::vector<std::array<int64_t, 3>>& xq) {
  for (int i : list) S.partners[i].clear();
  for (const auto& p : find_pairs(S, list, xq)) {
    S.partners[p.first].push_back(p.second);
    S.partners[p.second].push_back(p.first);
  }
  for (int i : list) std::sort(S.partners[i].begin(), S.partners[i].end());
}

// Searched voxels of the voxel range [lo, hi): the surface voxels, or every
// voxel in the "all voxels" scheme.
template <class R> static std::vector<int> searched(const Sim<R>& S, int lo, int hi) {
  std::vector<int> list;
  for (int i = lo; i < hi; ++i)
    if (S.prm.cand_all || S.T.surface[i]) list.push_back(i);
  return list;
}

// Shared world: every body's candidates at once (pairs may cross bodies).
template <class R> static void rebuild_world(Sim<R>& S) {
  auto xq = quantise_positions(S);
  for (int i = 0; i < S.T.N; ++i) S.partners[i].clear();
  search_pairs(S, searched(S, 0, S.T.N), xq);
  S.n_rebuilds++;
}

template <class R> static void rebuild_all_candidates(Sim<R>& S);

template <class R> static void rebuild_candidates(Sim<R>& S, int body) {
  const Topo& T = S.T;
  auto xq = quantise_positions(S);
  int lo = T.body_first[body], hi = T.body_first[body + 1];
  for (int i = lo; i < hi; ++i) S.partners[i].clear();
  search_pairs(S, searched(S, lo, hi), xq);
  S.n_rebuilds++;
}

template <class R> static double horizon_threshold(const Sim<R>& S) {
  // Rebuild once the accumulated relative motion could close the gap between
  // the 2-voxel horizon and the largest possible contact distance (equal to
  // half the horizon, one voxel, without actuation).
  double smax = 0.0;  // largest thermal strain any voxel can reach
  for (int v = 0; v < S.T.N; ++v) {
    double A, T0, ph;
    signal_of(S.prm, S.T.mat[v], &A, &T0, &ph);
    if (S.prm.act_P <= 0) A = 0.0;
    smax = std::max(smax, std::fabs(S.cte[v]) * (std::fabs(T0) + std::fabs(A)));
  }
  double cmax = S.T.l * (1.0 + smax);
  return 2.0 * S.T.l - cmax;
}

template <class R> static void rebuild_all_candidates(Sim<R>& S) {
  if (S.prm.collide_on == 2) rebuild_world(S);
  else for (int b = 0; b < S.T.n_bodies; ++b) rebuild_candidates(S, b);
}

// Folds one decision (step, voxel or pair, branch code) into the signature.
inline uint64_t fold_event(uint64_t h, long n, long a, long b, int code) {
  const uint64_t w[4] = {(uint64_t)n, (uint64_t)a, (uint64_t)b, (uint64_t)code};
  for (uint64_t x : w) { h ^= x; h *= 1099511628211ull; }
  return h;
}

// One synchronous step of every voxel (Sec 2.1: all forces, then all positions).
template <class R> static int step(Sim<R>& S) {
  const Topo& T = S.T;
  int N = T.N;
  std::vector<R> dT(N);
  for (int v = 0; v < N; ++v) dT[v] = delta_T(S, v);
  // (1) all bond forces
  S.bo.resize(T.bonds.size());
  for (size_t b = 0; b < T.bonds.size(); ++b) bond_force(S, (int)b, dT, S.bo[b]);
  // (2) per voxel: sum, external forces, contacts, floor/friction -> new momenta
  std::vector<V3<R>> Pn(S.P), phin(S.phi);
  std::vector<uint8_t> statn(S.stat);
  const Params& p = S.prm;
  double l = T.l;
  for (int v = 0; v < N; ++v) {
    if (S.fixed[v]) continue;
    double m = S.mass[v], I = S.inertia[v], dt = S.dt[T.body[v]];
    V3<R> F, M;
    for (int s = 0; s < 6; ++s) {  // fixed order -x,+x,-y,+y,-z,+z (Sec 2.1.2 sum)
      int id = T.slot_bond[v][s];
      if (id < 0) continue;
      if (s % 2 == 0) { F += S.bo[id].F2; M += S.bo[id].M2; }  // v is the bond's voxel 2
      else            { F += S.bo[id].F1; M += S.bo[id].M1; }  // v is the bond's voxel 1
    }
    F += V3<R>(R(S.Fext[v].x), R(S.Fext[v].y), R(S.Fext[v].z));
    F.z += R(m * p.gravity_z);                      // gravity (Sec 2.2.1)
    V3<R> vel = S.P[v] * R(1.0 / m), om = S.phi[v] * R(1.0 / I);
    R kv = S.E[v] * R(l);
    if (p.zeta_ground != 0.0) {                     // damping to ground (Sec 2.1.5)
      F -= vel * (R(2.0 * p.zeta_ground) * sqrt(R(m) * kv));
      M -= om * (R(2.0 * p.zeta_ground) * sqrt(R(I) * kv * R(l * l / 6.0)));
    }
    R h = R(0.5 * l) * (R(1.0) + R(S.cte[v]) * dT[v]);  // current half size
    if (p.collide_on) {                             // voxel-voxel contacts
      for (int j : S.partners[v]) {
        V3<R> d = S.D[j] - S.D[v];
        R r = sqrt(dot(d, d));
        R hj = R(0.5 * l) * (R(1.0) + R(S.cte[j]) * dT[j]);
        R c = h + hj;
        if (!(r < c)) continue;
        S.events = fold_event(S.events, S.n, v, j, 1);
        V3<R> nh = d * (R(1.0) / r);
        R kc = R(2.0) * S.E[v] * S.E[j] / (S.E[v] + S.E[j]) * R(l);
        // READING (force law not given): penalty spring on the overlap plus
        // normal damping with ratio zeta_c on the smaller mass.
        F -= nh * (kc * (c - r));
        V3<R> vj = S.P[j] * R(1.0 / S.mass[j]);
        double mmin = std::min(m, S.mass[j]);
        F += nh * (R(2.0 * p.zeta_collision) * sqrt(R(mmin) * kc) * dot(vj - vel, nh));
      }
    }
    V3<R> Pv = S.P[v];
    if (p.floor_on) {
      R pen = h - S.D[v].z;
      if (pen > R(0.0)) {
        R Fn = kv * pen;
        F.z += Fn - R(2.0 * p.zeta_collision) * sqrt(R(m) * kv) * vel.z;
        R Flx = F.x, Fly = F.y;
        R Fl = sqrt(Flx * Flx + Fly * Fly);
        R vl = sqrt(vel.x * vel.x + vel.y * vel.y);
        R mus = R(S.mus[v]) * Fn, mud = R(S.muk[v]) * Fn;
        bool zero_l = false;
        int branch;
        if (statn[v]) {
          if (Fl <= mus) { zero_l = true; branch = 2; }   // held by static friction
          else { statn[v] = 0; F.x -= mud * Flx / Fl; F.y -= mud * Fly / Fl; branch = 3; }
        } else {
          if (vl <= mud * R(dt / m) && Fl <= mus) { zero_l = true; statn[v] = 1; branch = 4; }  // halt
          else if (vl > R(0.0)) { F.x -= mud * vel.x / vl; F.y -= mud * vel.y / vl; branch = 5; }
          else { F.x -= mud * Flx / Fl; F.y -= mud * Fly / Fl; branch = 6; }
        }
        S.events = fold_event(S.events, S.n, v, -1, branch);
        if (zero_l) { F.x = R(0.0); F.y = R(0.0); Pv.x = R(0.0); Pv.y = R(0.0); }
      } else {
        statn[v] = 0;
      }
    }
    Pn[v] = Pv + F * R(dt);          // P_{n+1} = P_n + F dt
    phin[v] = S.phi[v] + M * R(dt);  // phi_{n+1} = phi_n + M dt
  }
  // (3) update all positions and orientations synchronously (Sec 2.1.3)
  std::vector<double> vmax(T.n_bodies, 0.0);
  for (int v = 0; v < N; ++v) {
    if (S.fixed[v]) continue;
    double dt = S.dt[T.body[v]];
    S.P[v] = Pn[v]; S.phi[v] = phin[v]; S.stat[v] = statn[v];
    S.D[v] += S.P[v] * R(dt / S.mass[v]);
    V3<R> w = S.phi[v] * R(dt / S.inertia[v]);
    S.q[v] = qnormalize(qmul(qexp_vec(w), S.q[v]));   // world-frame rotation
    V3<R> vel = S.P[v] * R(1.0 / S.mass[v]);
    double sp = std::sqrt(val(dot(vel, vel)));
    if (!std::isfinite(sp)) return -1;
    vmax[T.body[v]] = std::max(vmax[T.body[v]], sp);
  }
  S.n++;
  // (4) collision horizon (Sec 2.2.2); in the shared world one accumulator
  // over every body (relative motion between bodies counts too)
  if (p.collide_on && p.cand_every) {
    rebuild_all_candidates(S);
  } else if (p.collide_on == 2) {
    double vm = 0.0;
    for (int b = 0; b < T.n_bodies; ++b) vm = std::max(vm, vmax[b]);
    S.acc[0] += 2.0 * vm * S.dt[0];
    if (S.acc[0] >= horizon_threshold(S)) { rebuild_world(S); S.acc[0] = 0.0; }
  } else if (p.collide_on) {
    double thr = horizon_threshold(S);
    for (int b = 0; b < T.n_bodies; ++b) {
      S.acc[b] += 2.0 * vmax[b] * S.dt[b];
      if (S.acc[b] >= thr) { rebuild_candidates(S, b); S.acc[b] = 0.0; }
    }
  }
  return 0;
}

template <class R> static void reset_state(Sim<R>& S, const double* v0) {
  int N = S.T.N;
  S.D.resize(N); S.P.assign(N, V3<R>()); S.phi.assign(N, V3<R>());
  S.q.assign(N, Q4<R>()); S.stat.assign(N, 0);
  for (int v = 0; v < N; ++v) {
    V3<double> an = S.anchor(v);
    S.D[v] = V3<R>(R(an.x), R(an.y), R(an.z));
    if (v0 && !S.fixed[v]) S.P[v] = V3<R>(R(v0[0] * S.mass[v]), R(v0[1] * S.mass[v]), R(v0[2] * S.mass[v]));
  }
  S.n = 0;
  S.acc.assign(S.T.n_bodies, 0.0);
  S.partners.assign(N, {});
  S.events = 1469598103934665603ull;
}

// Elastic energy of the bonds: 1/2 u^T K u in each bond's reduced frame.
template <class R> static double elastic_energy(const Sim<R>& S) {
  std::vector<R> dT(S.T.N);
  for (int v = 0; v < S.T.N; ++v) dT[v] = delta_T(S, v);
  double U = 0.0;
  for (const auto& bd : S.T.bonds) {
    BeamK<R> k = beam_constants(S, bd.v1, bd.v2);
    R eps = R(0.5) * (R(S.cte[bd.v1]) * dT[bd.v1] + R(S.cte[bd.v2]) * dT[bd.v2]);
    V3<R> p = to_axis(qrot_inv(S.q[bd.v1], S.D[bd.v2] - S.D[bd.v1]), bd.axis);
    V3<R> th = to_axis(qlog_vec(qmul(qconj(S.q[bd.v1]), S.q[bd.v2])), bd.axis);
    double X = val(p.x) - S.T.l * (1.0 + val(eps)), Y = val(p.y), Z = val(p.z);
    double tx = val(th.x), ty = val(th.y), tz = val(th.z);
    double a1 = val(k.a1), a2 = val(k.a2), b1 = val(k.b1), b2 = val(k.b2), b3 = val(k.b3);
    U += 0.5 * (a1 * X * X + b1 * Y * Y + b1 * Z * Z + a2 * tx * tx + 2 * b3 * ty * ty + 2 * b3 * tz * tz)
         - b2 * Y * tz + b2 * Z * ty;
  }
  return U;
}

}  // namespace orc

// ---------------------------------------------------------------------------
// C interface (loaded with ctypes by the tests)
// ---------------------------------------------------------------------------
using namespace orc;

struct orc_sim {
  Sim<double> S;
  std::vector<double> logE;   // empty if not set
  Sim<Dual>* SD = nullptr;    // dual copy for directional derivatives
};

template <class R> static void init_sim(Sim<R>& S, int n_bodies, const int32_t* dims, const uint8_t* grid,
                                        double l, const double* pal, int n_mat, const double* origin) {
  build_topology(S.T, n_bodies, dims, grid, l);
  S.pal.assign(pal, pal + 6 * n_mat);
  S.n_mat = n_mat;
  S.origin.resize(n_bodies);
  for (int b = 0; b < n_bodies; ++b)
    S.origin[b] = origin ? V3<double>(origin[3 * b], origin[3 * b + 1], origin[3 * b + 2]) : V3<double>();
  int N = S.T.N;
  S.phase.assign(N, R(0.0));
  S.fixed.assign(N, 0);
  S.Fext.assign(N, V3<double>());
  quant_params(l, &S.qK, &S.qQ);
  set_materials(S, nullptr);
  compute_dt(S);
  reset_state(S, nullptr);
}

extern "C" {

orc_sim* orc_create(int n_bodies, const int32_t* dims, const uint8_t* grid, double l,
                    const double* palette, int n_mat, const double* origin) {
  for (int b = 0; b < n_bodies; ++b)
    if (dims[3 * b] < 1 || dims[3 * b + 1] < 1 || dims[3 * b + 2] < 1) return nullptr;
  orc_sim* o = new orc_sim();
  init_sim(o->S, n_bodies, dims, grid, l, palette, n_mat, origin);
  for (int v = 0; v < o->S.T.N; ++v)
    if (o->S.T.mat[v] >= n_mat) { delete o; return nullptr; }
  return o;
}

void orc_destroy(orc_sim* o) { if (o) { delete o->SD; delete o; } }

int orc_n_voxels(orc_sim* o) { return o->S.T.N; }
int orc_n_bonds(orc_sim* o) { return (int)o->S.T.bonds.size(); }

void orc_topology(orc_sim* o, int32_t* body_ijk /*N x 4*/, int32_t* nbr /*N x 6*/, uint8_t* surface) {
  const Topo& T = o->S.T;
  for (int v = 0; v < T.N; ++v) {
    if (body_ijk) { body_ijk[4 * v] = T.body[v]; body_ijk[4 * v + 1] = T.vi[v]; body_ijk[4 * v + 2] = T.vj[v]; body_ijk[4 * v + 3] = T.vk[v]; }
    if (nbr) for (int s = 0; s < 6; ++s) nbr[6 * v + s] = T.nbr[v][s];
    if (surface) surface[v] = T.surface[v];
  }
}

void orc_bonds(orc_sim* o, int32_t* out /*n_bonds x 3*/) {
  const Topo& T = o->S.T;
  for (size_t b = 0; b < T.bonds.size(); ++b) {
    out[3 * b] = T.bonds[b].v1; out[3 * b + 1] = T.bonds[b].v2; out[3 * b + 2] = T.bonds[b].axis;
  }
}

void orc_set_params(orc_sim* o, double zeta_bond, double zeta_ground, double zeta_collision, double gravity_z,
                    int floor_on, int collide_on, double act_A, long act_P, double act_T0, double dt_factor) {
  Params& p = o->S.prm;
  p.zeta_bond = zeta_bond; p.zeta_ground = zeta_ground; p.zeta_collision = zeta_collision;
  p.gravity_z = gravity_z; p.floor_on = floor_on; p.collide_on = collide_on;
  p.act_A = act_A; p.act_P = act_P; p.act_T0 = act_T0; p.dt_factor = dt_factor;
  compute_dt(o->S);
}

void orc_set_material_actuation(orc_sim* o, const double* amplitude, const double* offset, const double* phase) {
  Params& p = o->S.prm;
  const int nm = o->S.n_mat;
  if (amplitude) p.mat_A.assign(amplitude, amplitude + nm); else p.mat_A.clear();
  if (offset) p.mat_T0.assign(offset, offset + nm); else p.mat_T0.clear();
  if (phase) p.mat_ph.assign(phase, phase + nm); else p.mat_ph.clear();
}

void orc_set_collision_scheme(orc_sim* o, int all_voxels, int every_step) {
  o->S.prm.cand_all = all_voxels ? 1 : 0;
  o->S.prm.cand_every = every_step ? 1 : 0;
}

void orc_set_brute_search(orc_sim* o, int on) { o->S.prm.brute_search = on ? 1 : 0; }

void orc_set_voxel_params(orc_sim* o, const double* logE, const double* phase) {
  Sim<double>& S = o->S;
  if (logE) { o->logE.assign(logE, logE + S.T.N); set_materials(S, logE); compute_dt(S); }
  if (phase) for (int v = 0; v < S.T.N; ++v) S.phase[v] = phase[v];
}

void orc_set_fixed(orc_sim* o, const uint8_t* mask) {
  for (int v = 0; v < o->S.T.N; ++v) o->S.fixed[v] = mask[v] ? 1 : 0;
}

void orc_set_force(orc_sim* o, const double* F) {
  for (int v = 0; v < o->S.T.N; ++v) o->S.Fext[v] = V3<double>(F[3 * v], F[3 * v + 1], F[3 * v + 2]);
}

// Paper App. B, AddFixedRegion / AddForcedRegion: a voxel "touching" the region
// (fractions of the workspace) is selected.  READING: touching = the closed
// voxel cube [i/nx, (i+1)/nx] x ... overlaps the closed region box.
int orc_region_mask(orc_sim* o, int body, const double* loc, const double* size, uint8_t* mask) {
  const Topo& T = o->S.T;
  auto d = T.dims[body];
  int cnt = 0;
  for (int v = 0; v < T.N; ++v) {
    int c[3] = {T.vi[v], T.vj[v], T.vk[v]};
    bool in = T.body[v] == body;
    for (int a = 0; a < 3 && in; ++a) {
      double lo = (double)c[a] / d[a], hi = (double)(c[a] + 1) / d[a];
      if (hi < loc[a] || lo > loc[a] + size[a]) in = false;
    }
    mask[v] = in ? 1 : 0;
    cnt += in;
  }
  return cnt;
}

void orc_reset(orc_sim* o, const double* v0) {
  reset_state(o->S, v0);
  if (o->S.prm.collide_on) rebuild_all_candidates(o->S);
}

// Rebuild every body's collision candidates from the current positions.
void orc_reset_candidates(orc_sim* o) {
  rebuild_all_candidates(o->S);
  for (int b = 0; b < o->S.T.n_bodies; ++b) o->S.acc[b] = 0.0;
}

double orc_get_dt(orc_sim* o, int body) { return o->S.dt[body]; }
void orc_set_dt(orc_sim* o, int body, double dt) { o->S.dt[body] = dt; }
long orc_get_step(orc_sim* o) { return o->S.n; }

int orc_step(orc_sim* o, long n) {
  for (long i = 0; i < n; ++i)
    if (step(o->S) != 0) return -1;
  return 0;
}

// State in the API's layout: absolute position, quaternion (w,x,y,z),
// linear velocity, angular velocity, static-friction flag.
void orc_get_state(orc_sim* o, double* pos, double* quat, double* vel, double* angvel, uint8_t* stat) {
  Sim<double>& S = o->S;
  for (int v = 0; v < S.T.N; ++v) {
    if (pos) { pos[3 * v] = S.D[v].x; pos[3 * v + 1] = S.D[v].y; pos[3 * v + 2] = S.D[v].z; }
    if (quat) { quat[4 * v] = S.q[v].w; quat[4 * v + 1] = S.q[v].x; quat[4 * v + 2] = S.q[v].y; quat[4 * v + 3] = S.q[v].z; }
    if (vel) for (int a = 0; a < 3; ++a) vel[3 * v + a] = S.P[v][a] / S.mass[v];
    if (angvel) for (int a = 0; a < 3; ++a) angvel[3 * v + a] = S.phi[v][a] / S.inertia[v];
    if (stat) stat[v] = S.stat[v];
  }
}

void orc_set_state(orc_sim* o, const double* pos, const double* quat, const double* vel, const double* angvel,
                   const uint8_t* stat) {
  Sim<double>& S = o->S;
  for (int v = 0; v < S.T.N; ++v) {
    if (pos) S.D[v] = V3<double>(pos[3 * v], pos[3 * v + 1], pos[3 * v + 2]);
    if (quat) S.q[v] = Q4<double>(quat[4 * v], quat[4 * v + 1], quat[4 * v + 2], quat[4 * v + 3]);
    if (vel) S.P[v] = V3<double>(vel[3 * v] * S.mass[v], vel[3 * v + 1] * S.mass[v], vel[3 * v + 2] * S.mass[v]);
    if (angvel) S.phi[v] = V3<double>(angvel[3 * v] * S.inertia[v], angvel[3 * v + 1] * S.inertia[v], angvel[3 * v + 2] * S.inertia[v]);
    if (stat) S.stat[v] = stat[v];
  }
}

void orc_set_step_counter(orc_sim* o, long n) { o->S.n = n; }

// Forces on both voxels of one bond for the current state: F1, M1, F2, M2 (12 doubles).
void orc_bond_force(orc_sim* o, int id, double* out) {
  Sim<double>& S = o->S;
  std::vector<double> dT(S.T.N);
  for (int v = 0; v < S.T.N; ++v) dT[v] = delta_T(S, v);
  Sim<double>::BondOut b;
  bond_force(S, id, dT, b);
  V3<double>* vs[4] = {&b.F1, &b.M1, &b.F2, &b.M2};
  for (int i = 0; i < 4; ++i) for (int a = 0; a < 3; ++a) out[3 * i + a] = (*vs[i])[a];
}

void orc_energy(orc_sim* o, double* out /* KE_lin, KE_rot, U_elastic, U_gravity */) {
  Sim<double>& S = o->S;
  double kl = 0, kr = 0, ug = 0;
  for (int v = 0; v < S.T.N; ++v) {
    kl += 0.5 * dot(S.P[v], S.P[v]) / S.mass[v];
    kr += 0.5 * dot(S.phi[v], S.phi[v]) / S.inertia[v];
    ug -= S.mass[v] * S.prm.gravity_z * S.D[v].z;
  }
  out[0] = kl; out[1] = kr; out[2] = elastic_energy(S); out[3] = ug;
}

void orc_momentum(orc_sim* o, double* out /* P (3), L about origin (3) */) {
  Sim<double>& S = o->S;
  V3<double> P, L;
  for (int v = 0; v < S.T.N; ++v) { P += S.P[v]; L += cross(S.D[v], S.P[v]) + S.phi[v]; }
  for (int a = 0; a < 3; ++a) { out[a] = P[a]; out[3 + a] = L[a]; }
}

// Candidate pairs (i<j) of the current partner lists.
long orc_candidate_pairs(orc_sim* o, int32_t* pairs, long cap) {
  Sim<double>& S = o->S;
  long n = 0;
  for (int i = 0; i < S.T.N; ++i)
    for (int j : S.partners[i])
      if (j > i) { if (n < cap) { pairs[2 * n] = i; pairs[2 * n + 1] = j; } ++n; }
  return n;
}

long orc_n_rebuilds(orc_sim* o) { return o->S.n_rebuilds; }
// Signature of the discrete decisions since the last reset (see Sim::events).
uint64_t orc_event_signature(orc_sim* o) { return o->S.events; }
double orc_accumulator(orc_sim* o, int body) { return o->S.acc[body]; }

// Candidate pairs (i<j, sorted) for given anchor offsets o (N x 3 doubles,
// typically FP32 values widened exactly), searched body by body (all bodies
// at once in a shared world) with the search the simulator uses (the sweep,
// or brute force when set).
long orc_pairs_from_offsets(orc_sim* o, const double* off, int32_t* pairs, long cap) {
  Sim<double>& S = o->S;
  const Topo& T = S.T;
  std::vector<std::array<int64_t, 3>> xq(T.N);
  for (int v = 0; v < T.N; ++v) {
    int c[3] = {T.vi[v], T.vj[v], T.vk[v]};
    for (int a = 0; a < 3; ++a)
      xq[v][a] = (S.prm.collide_on == 2 ? (int64_t)std::nearbyint(std::ldexp(S.origin[T.body[v]][a], S.qK)) : 0) +
                 (int64_t)c[a] * S.qQ + (int64_t)std::nearbyint(std::ldexp(off[3 * v + a], S.qK));
  }
  std::vector<std::pair<int, int>> all;
  if (S.prm.collide_on == 2) {
    all = find_pairs(S, searched(S, 0, T.N), xq);
  } else {
    for (int b = 0; b < T.n_bodies; ++b) {
      auto p = find_pairs(S, searched(S, T.body_first[b], T.body_first[b + 1]), xq);
      all.insert(all.end(), p.begin(), p.end());
    }
  }
  std::sort(all.begin(), all.end());
  long n = 0;
  for (const auto& p : all) {
    if (n < cap) { pairs[2 * n] = p.first; pairs[2 * n + 1] = p.second; }
    ++n;
  }
  return n;
}

// Partners of one voxel i (all j != i, ascending) from offsets, by brute force.
long orc_partners_of(orc_sim* o, const double* off, int i, int32_t* out, long cap) {
  Sim<double>& S = o->S;
  const Topo& T = S.T;
  if (!S.prm.cand_all && !T.surface[i]) return 0;
  const bool world = S.prm.collide_on == 2;
  auto q = [&](int v, int a) {
    int c[3] = {T.vi[v], T.vj[v], T.vk[v]};
    return (world ? (int64_t)std::nearbyint(std::ldexp(S.origin[T.body[v]][a], S.qK)) : 0) +
           (int64_t)c[a] * S.qQ + (int64_t)std::nearbyint(std::ldexp(off[3 * v + a], S.qK));
  };
  long n = 0;
  for (int j = 0; j < T.N; ++j) {
    if (j == i || (!S.prm.cand_all && !T.surface[j])) continue;
    if (T.body[j] != T.body[i]) {
      if (!world) continue;
    } else {
      int man = std::abs(T.vi[i] - T.vi[j]) + std::abs(T.vj[i] - T.vj[j]) + std::abs(T.vk[i] - T.vk[j]);
      if (man <= 3) continue;
    }
    int64_t dx = q(i, 0) - q(j, 0), dy = q(i, 1) - q(j, 1), dz = q(i, 2) - q(j, 2);
    if (dx * dx + dy * dy + dz * dz < 4 * S.qQ * S.qQ) { if (n < cap) out[n] = j; ++n; }
  }
  return n;
}

void orc_quant_params(double l, int32_t* K, int64_t* Q) { int k; quant_params(l, &k, Q); *K = k; }

// ---- directional derivative of a rollout (forward mode) -------------------
// Runs the same rollout in dual numbers with logE and phase perturbed along
// (dlogE, dphase); returns the value and derivative of
// loss = sum over bodies of (x_CoM(n) - x_CoM(0)).
int orc_rollout_jvp(orc_sim* o, long n_steps, const double* dlogE, const double* dphase,
                    double* loss, double* dloss) {
  Sim<double>& S0 = o->S;
  Sim<Dual>* SD = new Sim<Dual>();
  SD->T = S0.T; SD->prm = S0.prm; SD->pal = S0.pal; SD->n_mat = S0.n_mat; SD->origin = S0.origin;
  SD->qK = S0.qK; SD->qQ = S0.qQ;
  int N = S0.T.N;
  // materials with dual log-stiffness
  SD->E.resize(N); SD->G.resize(N);
  SD->rho = S0.rho; SD->cte = S0.cte; SD->mus = S0.mus; SD->muk = S0.muk; SD->mass = S0.mass; SD->inertia = S0.inertia;
  for (int v = 0; v < N; ++v) {
    const double* m = &S0.pal[6 * S0.T.mat[v]];
    Dual le(o->logE.empty() ? std::log(m[0]) : o->logE[v], dlogE ? dlogE[v] : 0.0);
    SD->E[v] = exp(le);
    SD->G[v] = SD->E[v] / Dual(2.0 * (1.0 + m[1]));
  }
  SD->phase.resize(N);
  for (int v = 0; v < N; ++v) SD->phase[v] = Dual(S0.phase[v], dphase ? dphase[v] : 0.0);
  SD->fixed = S0.fixed; SD->Fext = S0.Fext;
  SD->dt = S0.dt;  // frozen timestep
  // current state of the double simulator as the starting point
  SD->D.resize(N); SD->P.resize(N); SD->phi.resize(N); SD->q.resize(N);
  for (int v = 0; v < N; ++v) {
    SD->D[v] = V3<Dual>(S0.D[v].x, S0.D[v].y, S0.D[v].z);
    SD->P[v] = V3<Dual>(S0.P[v].x, S0.P[v].y, S0.P[v].z);
    SD->phi[v] = V3<Dual>(S0.phi[v].x, S0.phi[v].y, S0.phi[v].z);
    SD->q[v] = Q4<Dual>(S0.q[v].w, S0.q[v].x, S0.q[v].y, S0.q[v].z);
  }
  SD->stat = S0.stat; SD->n = S0.n; SD->acc = S0.acc; SD->partners = S0.partners;
  std::vector<Dual> x0(S0.T.n_bodies, Dual(0.0)), msum(S0.T.n_bodies, Dual(0.0));
  for (int v = 0; v < N; ++v) { x0[S0.T.body[v]] += SD->D[v].x * Dual(S0.mass[v]); msum[S0.T.body[v]] += Dual(S0.mass[v]); }
  int rc = 0;
  for (long i = 0; i < n_steps && rc == 0; ++i) rc = step(*SD);
  Dual L(0.0);
  std::vector<Dual> x1(S0.T.n_bodies, Dual(0.0));
  for (int v = 0; v < N; ++v) x1[S0.T.body[v]] += SD->D[v].x * Dual(S0.mass[v]);
  for (int b = 0; b < S0.T.n_bodies; ++b) L += (x1[b] - x0[b]) / msum[b];
  *loss = L.v; *dloss = L.d;
  delete SD;
  return rc;
}

// ---- linear direct stiffness solve (static reference) ---------------------
// Assembles the paper's 12x12 beam matrix [K] (Sec 2.1.2) for every bond,
// rotated onto its lattice axis, and solves K u = f for the free DOFs with
// dense Gaussian elimination.  u, f: N x 6 (dx,dy,dz,rx,ry,rz).
// Assembles the global 6N x 6N stiffness of the lattice at rest from each
// bond's printed 12x12 [K] (Sec 2.1.2), rotated onto its lattice axis.
static void assemble_stiffness(const Sim<double>& S, std::vector<double>& K) {
  const Topo& T = S.T;
  int N = T.N, n = 6 * N;
  K.assign((size_t)n * n, 0.0);
  for (const auto& bd : T.bonds) {
    BeamK<double> k = beam_constants(S, bd.v1, bd.v2);
    double a1 = k.a1, a2 = k.a2, b1 = k.b1, b2 = k.b2, b3 = k.b3;
    // upper triangle of the printed matrix (row, col, value), 0-based
    double Ke[12][12] = {};
    auto set = [&](int r, int c, double x) { Ke[r][c] = x; Ke[c][r] = x; };
    set(0, 0, a1); set(0, 6, -a1);
    set(1, 1, b1); set(1, 5, b2); set(1, 7, -b1); set(1, 11, b2);
    set(2, 2, b1); set(2, 4, -b2); set(2, 8, -b1); set(2, 10, -b2);
    set(3, 3, a2); set(3, 9, -a2);
    set(4, 4, 2 * b3); set(4, 8, b2); set(4, 10, b3);
    set(5, 5, 2 * b3); set(5, 7, -b2); set(5, 11, b3);
    set(6, 6, a1);
    set(7, 7, b1); set(7, 11, -b2);
    set(8, 8, b1); set(8, 10, b2);
    set(9, 9, a2);
    set(10, 10, 2 * b3);
    set(11, 11, 2 * b3);
    // local DOF i of the element maps to global DOF of the voxel via Pi_a
    auto gdof = [&](int e) {
      int node = e / 6, w = e % 6, blk = w / 3, comp = w % 3;
      int gcomp = (comp + bd.axis) % 3;  // local[comp] = global[(comp+a)%3]
      int v = node == 0 ? bd.v1 : bd.v2;
      return 6 * v + 3 * blk + gcomp;
    };
    for (int r = 0; r < 12; ++r)
      for (int c = 0; c < 12; ++c) K[(size_t)gdof(r) * n + gdof(c)] += Ke[r][c];
  }
}

// Global stiffness (6N x 6N, DOFs x, y, z, rx, ry, rz per voxel) and the
// lumped mass of every DOF (m for translations, I = m l^2 / 6 for rotations):
// the linearised dynamics M u'' = -K u of the step at rest.
void orc_stiffness(orc_sim* o, double* K, double* mdiag) {
  Sim<double>& S = o->S;
  std::vector<double> Kv;
  assemble_stiffness(S, Kv);
  std::copy(Kv.begin(), Kv.end(), K);
  for (int v = 0; v < S.T.N; ++v)
    for (int d = 0; d < 6; ++d) mdiag[6 * v + d] = d < 3 ? S.mass[v] : S.inertia[v];
}

int orc_linear_static(orc_sim* o, const double* f, double* u) {
  Sim<double>& S = o->S;
  const Topo& T = S.T;
  int N = T.N, n = 6 * N;
  std::vector<double> K;
  assemble_stiffness(S, K);
  std::vector<int> free_dofs;
  for (int v = 0; v < N; ++v)
    if (!S.fixed[v]) for (int d = 0; d < 6; ++d) free_dofs.push_back(6 * v + d);
  int m = (int)free_dofs.size();
  std::vector<double> A((size_t)m * (m + 1));
  for (int r = 0; r < m; ++r) {
    for (int c = 0; c < m; ++c) A[(size_t)r * (m + 1) + c] = K[(size_t)free_dofs[r] * n + free_dofs[c]];
    A[(size_t)r * (m + 1) + m] = f[free_dofs[r]];
  }
  for (int c = 0; c < m; ++c) {  // Gaussian elimination with partial pivoting
    int piv = c;
    for (int r = c + 1; r < m; ++r)
      if (std::fabs(A[(size_t)r * (m + 1) + c]) > std::fabs(A[(size_t)piv * (m + 1) + c])) piv = r;
    if (std::fabs(A[(size_t)piv * (m + 1) + c]) < 1e-300) return -1;
    if (piv != c) for (int k = 0; k <= m; ++k) std::swap(A[(size_t)c * (m + 1) + k], A[(size_t)piv * (m + 1) + k]);
    for (int r = c + 1; r < m; ++r) {
      double fct = A[(size_t)r * (m + 1) + c] / A[(size_t)c * (m + 1) + c];
      if (fct == 0.0) continue;
      for (int k = c; k <= m; ++k) A[(size_t)r * (m + 1) + k] -= fct * A[(size_t)c * (m + 1) + k];
    }
  }
  std::vector<double> x(m);
  for (int r = m - 1; r >= 0; --r) {
    double s = A[(size_t)r * (m + 1) + m];
    for (int k = r + 1; k < m; ++k) s -= A[(size_t)r * (m + 1) + k] * x[k];
    x[r] = s / A[(size_t)r * (m + 1) + r];
  }
  for (int i = 0; i < n; ++i) u[i] = 0.0;
  for (int r = 0; r < m; ++r) u[free_dofs[r]] = x[r];
  return 0;
}

}  // extern "C"

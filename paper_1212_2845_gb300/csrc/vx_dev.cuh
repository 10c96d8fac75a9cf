// Device data layout and FP32 math of one explicit lattice step.
//
// All per-voxel arrays are in the internal order (bricks along a Morton
// curve, see vx_host.h).  The state of `pitch` voxels is three float4 planes
// and one float plane (13 floats, 52 bytes per voxel):
//   A = (offset x, y, z, quat w)   B = (quat x, y, z, vel x)
//   C = (vel y, z, angvel x, y)    D = angvel z
// so a warp moves a voxel's state in four coalesced vector accesses.  The
// state is double-buffered: a step reads st_in and writes st_out, so
// neighbours always see the state at step n.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace vx {

// State components in plane order (component c of voxel v lives at
// state_index(c, v, pitch) floats from the buffer start).
enum Comp { OX = 0, OY, OZ, QW, QX, QY, QZ, VX, VY, VZ, WX, WY, WZ, NPLANE };

__host__ __device__ __forceinline__ int64_t state_index(int c, int64_t v, int64_t pitch) {
  return c < 12 ? (int64_t)(c >> 2) * 4 * pitch + 4 * v + (c & 3) : 12 * pitch + v;
}

// Per-material constants precomputed on the host in double precision.
struct DevMat {
  float E;        // elastic modulus [Pa]
  float g_ratio;  // G / E = 1 / (2 (1 + nu))
  float cte;      // thermal expansion [1/K]
  float mu_s, mu_k;
  float m, inv_m; // rho l^3 and its inverse
  float I, inv_I; // m l^2 / 6 (solid cube) and its inverse
  // this material's temperature signal (Sec 2.3: several independent
  // "temperatures" may drive different materials): dT = act_T0 + act_A
  // sin(2 pi n / P + phase_voxel + act_phase); the global signal by default
  float act_A, act_T0, act_phase;
};

constexpr int kCandCap = 48;        // collision candidates per surface voxel
constexpr int kStatusUnstable = 1;  // status word bits
constexpr int kStatusCapacity = 2;
constexpr int kStatusTimeout = 4;   // a bounded device wait gave up
constexpr int kStatusArg = 8;       // an input value checked on the device was out of range
constexpr int kStatusBounds = 16;   // debug builds: an index failed its bounds check

// Bounds-checked debug builds (VX_BOUNDS_CHECK defined at compile time) test
// the indices that come from device tables before they are used: halo and
// bond staging slots, neighbour and candidate lists, hash buckets, cluster
// slices.  A failed check sets kStatusBounds, records the check site and the
// index in status[4] and status[5] (first failure only), and the caller skips
// the access; nothing traps.  Normal builds compile the checks away.
enum BoundsSite { kSiteHalo = 1, kSitePlusSlot, kSiteHaloBond, kSiteContact, kSiteBucket, kSiteSorted,
                  kSiteCluster };
#ifdef VX_BOUNDS_CHECK
__device__ __forceinline__ bool vx_in_bounds(int* status, long long i, long long n, int site) {
  if (i >= 0 && i < n) return true;
  if (!(atomicOr(status, kStatusBounds) & kStatusBounds)) {
    status[4] = site;
    status[5] = (int)i;
  }
  return false;
}
#define VX_IN_BOUNDS(status, i, n, site) ::vx::vx_in_bounds((status), (long long)(i), (long long)(n), (site))
#else
#define VX_IN_BOUNDS(status, i, n, site) true
#endif

// Phase angle of the actuation signal at step n (Sec 2.3), 2 pi (n mod P) / P,
// formed in FP32 as (n mod P) times c = fl(2 pi / P) with one rounding: the
// host (per-step launches) and the device (multi-step, batched and resident
// launches) get the same bits, and no FP64 runs on the GPU.
__host__ __device__ __forceinline__ float act_angle(int64_t step, int64_t P, float c) {
  if (P <= 0) return 0.f;
#ifdef __CUDA_ARCH__
  return __fmul_rn((float)(step % P), c);
#else
  return (float)(step % P) * c;
#endif
}

struct StepArgs {
  int N;
  int64_t pitch;
  float l;
  const float* st_in;      // NPLANE planes, state at step n
  float* st_out;           // NPLANE planes, state at step n + 1
  uint8_t* flags;          // bit 0 fixed, bit 1 static friction (updated in place by the owner)
  const uint8_t* mat;
  const uint32_t* lat;     // packed i | j << 11 | k << 22
  const int32_t* body;     // per voxel body, or nullptr for a single body
  const float* phase;      // per voxel or nullptr
  const float* logE;       // per voxel or nullptr
  const float* fext;       // 3 planes or nullptr
  const DevMat* mats;
  int n_mats;
  const float* lut;        // per material pair (a1, a2, b2, b3, c, cr, 0, 0), or nullptr
  const float* dt_body;    // per body
  const float* origin;     // 3 per body
  float zb, zg, zc, gz;
  int floor_on, collide_on;
  int act_on;              // temperature offset is non-zero somewhere
  float actA, actT0, act_w;  // global signal (materials carry their own copy); act_w = act_angle(n, P, c)
  int64_t step;
  // two-pass form
  const int32_t* nbr;      // 6 planes (-x,+x,-y,+y,-z,+z), internal indices
  float* bf;               // bond results: 9 components x 3 axes planes
  // fused form
  const int4* tile_a;      // v0, n_owned, halo start, n_halo
  const int4* tile_b;      // halo-bond list start, end
  const int32_t* halo;
  const uint16_t* plus;    // 3 planes: staging slot of the +a neighbour or 0xFFFF
  const uint32_t* hbonds;  // halo bonds: slot 1 | slot 2 << 12 | axis << 24
  const uint8_t* mask;     // per voxel 6-bit bond existence
  int n_tiles, max_local;
  // pipelined form
  const int32_t* tdesc;    // 8 ints per tile: v0, n_owned, n_halo, halo-bond start, n_halo_bonds
  const int32_t* hfix;     // halo indices at hfix[t * hstride + j]
  int hstride;
  const uint32_t* vw;      // per voxel: material | bond mask << 8
  const uint2* plus2;      // per voxel: +x | +y << 16, +z partner staging slots
  // collisions
  const int32_t* sidx;     // per voxel: surface index or -1
  const int32_t* ccount;   // per surface voxel
  const int32_t* vcnt;     // per voxel: candidate count (0 for voxels outside the search)
  const int32_t* cand;     // per surface voxel, kCandCap slots (internal indices, ascending)
  unsigned* vmax_bits;     // per body, float bits of max |v|
  int* status;             // [0] bits, [1] first bad voxel (internal), [2..3] step, [4..5] bounds site, index
  float* fm_out;           // 6 planes: bond force and moment sum of every voxel, or nullptr
  // collision horizon kept by the pipelined step itself (nullptr h_done: a
  // separate launch keeps it): the last CTA to finish updates the per-body
  // accumulators and flags the bodies to rebuild
  unsigned* h_done;        // CTAs done in this launch (0 between launches)
  float* h_acc;            // per body, or one for a shared world
  int* h_flag;             // per body: rebuild
  int* h_any;              // some body flagged
  float h_threshold;
  int h_world, n_bodies;
};


// ---------------------------------------------------------------------------
// small vector / quaternion helpers (FP32)
//
// Every operation is an explicit round-to-nearest intrinsic, so the compiler
// cannot fuse multiply-adds differently at different call sites: a bond or a
// voxel update gives the same bits wherever it is evaluated (own bond or halo
// bond, any tile size, fused or two-pass form).
// ---------------------------------------------------------------------------
struct V3f { float x, y, z; };
struct Qf { float w, x, y, z; };

__device__ __forceinline__ float fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float mul_(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float add_(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub_(float a, float b) { return __fsub_rn(a, b); }

__device__ __forceinline__ V3f v3(float a, float b, float c) { V3f r; r.x = a; r.y = b; r.z = c; return r; }
__device__ __forceinline__ V3f add(V3f a, V3f b) { return v3(add_(a.x, b.x), add_(a.y, b.y), add_(a.z, b.z)); }
__device__ __forceinline__ V3f sub(V3f a, V3f b) { return v3(sub_(a.x, b.x), sub_(a.y, b.y), sub_(a.z, b.z)); }
__device__ __forceinline__ V3f scl(V3f a, float s) { return v3(mul_(a.x, s), mul_(a.y, s), mul_(a.z, s)); }
// a + s b
__device__ __forceinline__ V3f axpy(V3f a, float s, V3f b) { return v3(fma_(s, b.x, a.x), fma_(s, b.y, a.y), fma_(s, b.z, a.z)); }
__device__ __forceinline__ float dot3(V3f a, V3f b) { return fma_(a.x, b.x, fma_(a.y, b.y, mul_(a.z, b.z))); }
__device__ __forceinline__ V3f cross3(V3f a, V3f b) {
  return v3(fma_(a.y, b.z, -mul_(a.z, b.y)), fma_(a.z, b.x, -mul_(a.x, b.z)), fma_(a.x, b.y, -mul_(a.y, b.x)));
}
// cyclic permutation taking lattice axis a to local x: local[i] = v[(i + a) % 3]
// (a is a compile-time constant in the unrolled callers, a register value
// where one code path serves all three axes)
__device__ __forceinline__ V3f to_axis_r(V3f v, int a) {
  return a == 0 ? v : (a == 1 ? v3(v.y, v.z, v.x) : v3(v.z, v.x, v.y));
}
__device__ __forceinline__ V3f from_axis_r(V3f u, int a) {
  return a == 0 ? u : (a == 1 ? v3(u.z, u.x, u.y) : v3(u.y, u.z, u.x));
}
template <int a> __device__ __forceinline__ V3f to_axis(V3f v) { return to_axis_r(v, a); }
template <int a> __device__ __forceinline__ V3f from_axis(V3f u) { return from_axis_r(u, a); }
// sqrt(x) for x > 0 from the hardware reciprocal square root (2 ulp)
__device__ __forceinline__ float fsqrt(float x) { return mul_(x, rsqrtf(x)); }

// Rotation matrix rows of unit quaternion q (body -> world).
struct M3f { V3f r0, r1, r2; };
__device__ __forceinline__ M3f qmat(Qf q) {
  float x2 = add_(q.x, q.x), y2 = add_(q.y, q.y), z2 = add_(q.z, q.z);
  float xx = mul_(q.x, x2), yy = mul_(q.y, y2), zz = mul_(q.z, z2);
  float xy = mul_(q.x, y2), xz = mul_(q.x, z2), yz = mul_(q.y, z2);
  float wx = mul_(q.w, x2), wy = mul_(q.w, y2), wz = mul_(q.w, z2);
  M3f m;
  m.r0 = v3(sub_(1.f, add_(yy, zz)), sub_(xy, wz), add_(xz, wy));
  m.r1 = v3(add_(xy, wz), sub_(1.f, add_(xx, zz)), sub_(yz, wx));
  m.r2 = v3(sub_(xz, wy), add_(yz, wx), sub_(1.f, add_(xx, yy)));
  return m;
}
__device__ __forceinline__ V3f mul(const M3f& m, V3f v) { return v3(dot3(m.r0, v), dot3(m.r1, v), dot3(m.r2, v)); }
__device__ __forceinline__ V3f mulT(const M3f& m, V3f v) {
  return v3(fma_(m.r0.x, v.x, fma_(m.r1.x, v.y, mul_(m.r2.x, v.z))),
            fma_(m.r0.y, v.x, fma_(m.r1.y, v.y, mul_(m.r2.y, v.z))),
            fma_(m.r0.z, v.x, fma_(m.r1.z, v.y, mul_(m.r2.z, v.z))));
}
// (R^T e_a) - e_a: row a of R(q) minus the unit vector, diagonal entry formed
// as -2 (sum of the other two squares) so that no cancellation occurs.
__device__ __forceinline__ V3f row_dev_r(const M3f& R, Qf q, int a) {
  if (a == 0) return v3(mul_(-2.f, fma_(q.y, q.y, mul_(q.z, q.z))), R.r0.y, R.r0.z);
  if (a == 1) return v3(R.r1.x, mul_(-2.f, fma_(q.x, q.x, mul_(q.z, q.z))), R.r1.z);
  return v3(R.r2.x, R.r2.y, mul_(-2.f, fma_(q.x, q.x, mul_(q.y, q.y))));
}
template <int a> __device__ __forceinline__ V3f row_dev(const M3f& R, Qf q) { return row_dev_r(R, q, a); }

// Rotation vector of conj(q1) * q2 (shortest arc).
__device__ __forceinline__ V3f rel_rotvec(Qf a, Qf b) {
  float w = fma_(a.w, b.w, fma_(a.x, b.x, fma_(a.y, b.y, mul_(a.z, b.z))));
  float x = fma_(a.w, b.x, fma_(-a.x, b.w, fma_(-a.y, b.z, mul_(a.z, b.y))));
  float y = fma_(a.w, b.y, fma_(a.x, b.z, fma_(-a.y, b.w, -mul_(a.z, b.x))));
  float z = fma_(a.w, b.z, fma_(-a.x, b.y, fma_(a.y, b.x, -mul_(a.z, b.w))));
  // shortest arc: for w < 0 the factor below takes the sign of w, which is
  // the rotation vector of -q (the same rotation)
  float s2 = fma_(x, x, fma_(y, y, mul_(z, z)));
  float f;
  if (s2 < mul_(0.04f, mul_(w, w))) {
    // 2 atan(t) / (t |w|) sign(w), t = s / |w| < 0.2: alternating series to
    // t^10 (remainder below t^12 / 13 < 4e-10); 1/w carries the sign
    float iw = __fdividef(1.f, w);
    float t2 = mul_(s2, mul_(iw, iw));
    float pz = fma_(t2, 1.f / 11.f, -1.f / 9.f);
    pz = fma_(t2, pz, 1.f / 7.f);
    pz = fma_(t2, pz, -0.2f);
    pz = fma_(t2, pz, 1.f / 3.f);
    f = mul_(add_(iw, iw), fma_(-t2, pz, 1.f));
  } else {
    float sq = sqrtf(s2);
    f = __fdividef(mul_(2.f, atan2f(sq, fabsf(w))), sq);
    if (w < 0.f) f = -f;
  }
  return v3(mul_(x, f), mul_(y, f), mul_(z, f));
}

// q <- normalize(exp(w dt) * q), w in the world frame
__device__ __forceinline__ Qf integrate_rot(Qf q, V3f w, float dt) {
  float a2 = mul_(dot3(w, w), mul_(dt, dt));
  float h2 = mul_(0.25f, a2);  // (|w| dt / 2)^2
  float c, k;                  // cos(|w|dt/2), sin(|w|dt/2)/|w|
  if (h2 < 1e-4f) {
    // series; remainders below h2^3 / 720 and h2^3 / 5040 relative (< 1.4e-15)
    c = fma_(h2, fma_(h2, 1.f / 24.f, -0.5f), 1.f);
    k = mul_(mul_(0.5f, dt), fma_(h2, fma_(h2, 1.f / 120.f, -1.f / 6.f), 1.f));
  } else {
    float a = sqrtf(a2);
    float sn, cs;
    sincosf(mul_(0.5f, a), &sn, &cs);
    c = cs;
    k = __fdividef(mul_(sn, dt), a);
  }
  Qf d;
  d.w = c; d.x = mul_(w.x, k); d.y = mul_(w.y, k); d.z = mul_(w.z, k);
  Qf r;
  r.w = fma_(d.w, q.w, fma_(-d.x, q.x, fma_(-d.y, q.y, -mul_(d.z, q.z))));
  r.x = fma_(d.w, q.x, fma_(d.x, q.w, fma_(d.y, q.z, -mul_(d.z, q.y))));
  r.y = fma_(d.w, q.y, fma_(-d.x, q.z, fma_(d.y, q.w, mul_(d.z, q.x))));
  r.z = fma_(d.w, q.z, fma_(d.x, q.y, fma_(-d.y, q.x, mul_(d.z, q.w))));
  float n = rsqrtf(fma_(r.w, r.w, fma_(r.x, r.x, fma_(r.y, r.y, mul_(r.z, r.z)))));
  r.w = mul_(r.w, n); r.x = mul_(r.x, n); r.y = mul_(r.y, n); r.z = mul_(r.z, n);
  return r;
}

struct VoxS { V3f o; Qf q; V3f v; V3f w; };

__device__ __forceinline__ VoxS unpack_vox(float4 a, float4 b, float4 c, float d) {
  VoxS s;
  s.o = v3(a.x, a.y, a.z);
  s.q.w = a.w; s.q.x = b.x; s.q.y = b.y; s.q.z = b.z;
  s.v = v3(b.w, c.x, c.y);
  s.w = v3(c.z, c.w, d);
  return s;
}

// State access on a buffer of `pitch` voxels (global or shared memory).
struct StPtr {
  float4* A; float4* B; float4* C; float* D;
  __device__ __forceinline__ StPtr(float* base, int64_t pitch) {
    A = reinterpret_cast<float4*>(base);
    B = A + pitch;
    C = B + pitch;
    D = reinterpret_cast<float*>(C + pitch);
  }
  __device__ __forceinline__ VoxS load(int64_t i) const { return unpack_vox(A[i], B[i], C[i], D[i]); }
  __device__ __forceinline__ void store(int64_t i, const VoxS& s) const {
    A[i] = make_float4(s.o.x, s.o.y, s.o.z, s.q.w);
    B[i] = make_float4(s.q.x, s.q.y, s.q.z, s.v.x);
    C[i] = make_float4(s.v.y, s.v.z, s.w.x, s.w.y);
    D[i] = s.w.z;
  }
};

__device__ __forceinline__ VoxS load_vox(const float* st, int64_t pitch, int64_t i) {
  return StPtr(const_cast<float*>(st), pitch).load(i);
}
__device__ __forceinline__ void store_vox(float* st, int64_t pitch, int64_t i, const VoxS& s) {
  StPtr(st, pitch).store(i, s);
}

// Thermal strain alpha dT of a voxel of material d with actuation phase ph
// at the current step (Sec 2.3), the material's own temperature signal.  The
// sine argument is reduced to [-pi, pi] for the hardware sine (absolute
// error below 4e-7); every product is rounded explicitly so that every
// caller gets the same bits whether it stores the value or uses it at once.
__device__ __forceinline__ float strain_of(const StepArgs& A, const DevMat& d, float ph) {
  if (!A.act_on) return 0.f;
  float x = __fadd_rn(__fadd_rn(A.act_w, ph), d.act_phase);
  x = __fmaf_rn(-6.28318530717958648f, rintf(__fmul_rn(x, 0.159154943091895336f)), x);
  return __fmul_rn(d.cte, __fmaf_rn(d.act_A, __sinf(x), d.act_T0));
}

__device__ __forceinline__ float thermal_strain(const StepArgs& A, int64_t g, const DevMat& d) {
  return strain_of(A, d, A.phase ? A.phase[g] : 0.f);
}

__device__ __forceinline__ float voxel_E(const StepArgs& A, int64_t g, int m) {
  return A.logE ? expf(A.logE[g]) : A.mats[m].E;
}

// Result of one bond: force on voxel 1 (voxel 2 gets -F1), moments on both.
struct BondOut { V3f F1, M1, M2; };

// Beam constants of a bond (Sec 2.1.2) and its damping coefficients (Sec 2.1.5).
// c2 = c / 2, c4 = c / 4, cr2 = cr / 2 with c = 2 zeta sqrt(m_min a1) and
// cr = 2 zeta sqrt(I_min b3) the translational and rotational damping coefficients.
struct BondK { float a1, a2, b2, b3, c2, c4, cr2; };  // b1 = a1 for cubic voxels

__device__ __forceinline__ BondK bond_consts(float l, float E1, float E2, float G1, float G2, float mmin, float Imin,
                                             float zb) {
  float Ec = __fdividef(mul_(mul_(2.f, E1), E2), add_(E1, E2));
  float Gc = __fdividef(mul_(mul_(2.f, G1), G2), add_(G1, G2));
  const float l2 = mul_(l, l), l3 = mul_(l2, l);
  BondK k;
  k.a1 = mul_(Ec, l);                      // E_c A / l
  k.a2 = mul_(mul_(Gc, l3), 1.f / 6.f);    // G_c J / l
  k.b2 = mul_(mul_(Ec, l2), 0.5f);         // 6 E_c I / l^2
  k.b3 = mul_(mul_(Ec, l3), 1.f / 6.f);    // 2 E_c I / l
  const float c = mul_(mul_(2.f, zb), fsqrt(mul_(mmin, k.a1)));
  k.c2 = mul_(c, 0.5f);
  k.c4 = mul_(c, 0.25f);
  k.cr2 = mul_(zb, fsqrt(mul_(Imin, k.b3)));
  return k;
}

__device__ __forceinline__ BondK lut_consts(const float* lut, int n_mats, int m1, int m2) {
  const float4* e = reinterpret_cast<const float4*>(lut) + 2 * (m1 * n_mats + m2);
  float4 u = e[0], w = e[1];
  BondK k;
  k.a1 = u.x; k.a2 = u.y; k.b2 = u.z; k.b3 = u.w; k.c2 = w.x; k.c4 = w.y; k.cr2 = w.z;
  return k;
}

// One bond along lattice axis a from voxel 1 (negative side) to voxel 2:
// co-rotational beam (Sec 2.1.2) in voxel 1's frame (R1 = R(q1)), local
// damping (Sec 2.1.5), rest length scaled by the mean thermal strain (Sec 2.3).
__device__ __forceinline__ BondOut bond_eval_r(const VoxS& s1, const M3f& R1, const VoxS& s2, float l,
                                               const BondK& k, float eps, bool damp, int a) {
  const float a1 = k.a1, a2 = k.a2, b1 = k.a1, b2 = k.b2, b3 = k.b3;
  // position of voxel 2 in voxel 1's frame minus its rest vector l e_a:
  // R1^T (l e_a + do) - l e_a = R1^T do + l (R1^T e_a - e_a)
  V3f dO = sub(s2.o, s1.o);
  V3f p = to_axis_r(axpy(mulT(R1, dO), l, row_dev_r(R1, s1.q, a)), a);
  float X = fma_(-l, eps, p.x), Y = p.y, Z = p.z;
  V3f th = to_axis_r(rel_rotvec(s1.q, s2.q), a);
  // bond forces on the voxels: the negated rows of [K] u (reduced form)
  V3f F1 = v3(mul_(a1, X), fma_(b1, Y, -mul_(b2, th.z)), fma_(b1, Z, mul_(b2, th.y)));
  V3f M1 = v3(mul_(a2, th.x), fma_(-b2, Z, -mul_(b3, th.y)), fma_(b2, Y, -mul_(b3, th.z)));
  const float b3x2 = add_(b3, b3);
  V3f M2 = v3(-mul_(a2, th.x), fma_(-b2, Z, -mul_(b3x2, th.y)), fma_(b2, Y, -mul_(b3x2, th.z)));
  BondOut o;
  o.F1 = mul(R1, from_axis_r(F1, a));
  o.M1 = mul(R1, from_axis_r(M1, a));
  o.M2 = mul(R1, from_axis_r(M2, a));
  if (damp) {
    // V_{2->1} = (v2 - Va) + (D2 - Da) x wa = (v2 - v1)/2 + (l e_a + do) x (w1 + w2)/4;
    // F1 += c V_{2->1};  M1 += cr (w2 - wa) = cr/2 (w2 - w1);  M2 -= the same
    V3f r = dO;
    if (a == 0) r.x = add_(r.x, l); else if (a == 1) r.y = add_(r.y, l); else r.z = add_(r.z, l);
    const V3f rw = cross3(r, add(s1.w, s2.w));
    o.F1 = axpy(axpy(o.F1, k.c2, sub(s2.v, s1.v)), k.c4, rw);
    const V3f dw = sub(s2.w, s1.w);
    o.M1 = axpy(o.M1, k.cr2, dw);
    o.M2 = axpy(o.M2, -k.cr2, dw);
  }
  return o;
}

template <int a>
__device__ __forceinline__ BondOut bond_eval(const VoxS& s1, const M3f& R1, const VoxS& s2, float l, const BondK& k,
                                             float eps, bool damp) {
  return bond_eval_r(s1, R1, s2, l, k, eps, damp, a);
}

// Stores the bond force and moment sums of voxel v when the caller asked for
// them (the adjoint form records them while it recomputes a segment).
__device__ __forceinline__ void store_bond_sums(const StepArgs& A, int64_t v, V3f F, V3f M) {
  if (!A.fm_out) return;
  float* o = A.fm_out + v;
  const int64_t P = A.pitch;
  o[0] = F.x; o[P] = F.y; o[2 * P] = F.z; o[3 * P] = M.x; o[4 * P] = M.y; o[5 * P] = M.z;
}

__device__ __forceinline__ void record_bad(const StepArgs& A, int v) {
  if (atomicOr(&A.status[0], kStatusUnstable) & kStatusUnstable) return;
  A.status[1] = v;
  *reinterpret_cast<long long*>(&A.status[2]) = (long long)A.step;
}

// Grid-wide barrier of a cooperative launch (every CTA co-resident).  The
// last CTA to arrive resets the count and releases the generation; the others
// poll it, busily for the first few hundred polls (CTAs of one launch arrive
// within microseconds) and then with short naps, for at most a budget of
// max_spins x 128 SM clock cycles (2^24: about a second at 2 GHz).  Returns
// false (and sets the timeout status bit) if the wait gave up, after which
// the caller ends the launch.  Every thread then performs its own acquire,
// so its later loads (including cp.async) see every write released before
// the barrier.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned n_ctas, long long max_spins, int* status) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    unsigned gen, prev, now;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(gen) : "l"(bar + 1) : "memory");
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(prev) : "l"(bar) : "memory");
    if (prev + 1 == n_ctas) {
      asm volatile("st.relaxed.gpu.global.u32 [%0], 0;" ::"l"(bar) : "memory");
      asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar + 1) : "memory");
    } else {
      const long long t0 = clock64(), budget = max_spins * 128;
      for (int it = 0;; ++it) {
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(now) : "l"(bar + 1) : "memory");
        if (now != gen) break;
        if (clock64() - t0 > budget) {
          atomicOr(status, kStatusTimeout);
          ok = 0;
          break;
        }
        if (it >= 256) __nanosleep(32);
      }
    }
  }
  __syncthreads();
  asm volatile("{\n .reg .u32 t;\n ld.acquire.gpu.global.u32 t, [%0];\n}" ::"l"(bar + 1) : "memory");
  return ok != 0;
}

// Per-voxel inputs of the voxel update, loaded before the bond phase so the
// update itself issues no dependent global reads.
struct VoxMeta {
  uint32_t lat;   // packed lattice coordinate
  int m;          // material
  int b;          // body
  uint8_t fl;     // flags
  float dt, z0;   // body timestep, anchor height of the voxel centre
  V3f fext;
  int nc;         // collision candidates of the voxel (0 with collisions off)
};

__device__ __forceinline__ VoxMeta load_meta(const StepArgs& A, int v) {
  VoxMeta mt;
  mt.lat = A.lat[v];
  mt.m = A.mat[v];
  mt.b = A.body ? A.body[v] : 0;
  mt.fl = A.flags[v];
  mt.dt = A.dt_body[mt.b];
  mt.z0 = fma_(add_((float)(int)(mt.lat >> 22), 0.5f), A.l, A.origin[3 * mt.b + 2]);
  const int64_t P = A.pitch;
  mt.fext = A.fext ? v3(A.fext[v], A.fext[P + v], A.fext[2 * P + v]) : v3(0.f, 0.f, 0.f);
  mt.nc = A.collide_on ? A.vcnt[v] : 0;
  return mt;
}

// Everything a voxel does after its bond forces are summed (Sec 2.2.1,
// Sec 2.2.2, Sec 2.1.3): external force, gravity, ground damping, voxel
// contacts, floor contact with Coulomb friction, then integration.  Updates
// s and fl (the caller stores them); returns |v| for the collision horizon.
__device__ __forceinline__ float voxel_update(const StepArgs& A, int v, const VoxMeta& mt, VoxS& s, uint8_t& fl,
                                              V3f F, V3f M, float adT, float Ev, const DevMat* mats) {
  const int64_t P = A.pitch;
  fl = mt.fl;
  if (fl & 1u) return 0.f;  // fixed: immobile, state carried over
  const DevMat& d = mats[mt.m];
  const float dt = mt.dt;
  const float l = A.l;
  F = add(F, mt.fext);
  F.z = fma_(d.m, A.gz, F.z);
  float kv = mul_(Ev, l);
  if (A.zg != 0.f) {
    F = axpy(F, -mul_(mul_(2.f, A.zg), fsqrt(mul_(d.m, kv))), s.v);
    M = axpy(M, -mul_(mul_(2.f, A.zg), fsqrt(mul_(mul_(d.I, kv), mul_(mul_(l, l), 1.f / 6.f)))), s.w);
  }
  const float hl = mul_(0.5f, l);
  float h = fma_(hl, adT, hl);  // current half size l (1 + adT) / 2
  if (A.collide_on && mt.nc > 0) {
    // the list is read only for a voxel that has candidates (most have none)
    const int si = A.sidx[v];
    if (si >= 0) {
      const uint32_t lp = mt.lat;
      int vi = (int)(lp & 2047u), vj = (int)((lp >> 11) & 2047u), vk = (int)(lp >> 22);
      const int nc = mt.nc;
      const int32_t* cl = A.cand + (int64_t)si * kCandCap;
      for (int c = 0; c < nc; ++c) {
        int j = cl[c];
        if (!VX_IN_BOUNDS(A.status, j, A.N, kSiteContact)) continue;
        uint32_t lq = A.lat[j];
        const StPtr sp(const_cast<float*>(A.st_in), P);
        const float4 ja = sp.A[j], jb = sp.B[j], jc = sp.C[j];
        V3f dd = v3(fma_((float)((int)(lq & 2047u) - vi), l, sub_(ja.x, s.o.x)),
                    fma_((float)((int)((lq >> 11) & 2047u) - vj), l, sub_(ja.y, s.o.y)),
                    fma_((float)((int)(lq >> 22) - vk), l, sub_(ja.z, s.o.z)));
        if (A.body) {  // a partner of another body (shared world): add the origins' difference
          const int bj = A.body[j];
          if (bj != mt.b)
            dd = add(dd, v3(sub_(A.origin[3 * bj], A.origin[3 * mt.b]), sub_(A.origin[3 * bj + 1], A.origin[3 * mt.b + 1]),
                            sub_(A.origin[3 * bj + 2], A.origin[3 * mt.b + 2])));
        }
        float r2 = dot3(dd, dd);
        int mj = A.mat[j];
        const DevMat& dj = mats[mj];
        float hj = fma_(hl, thermal_strain(A, j, dj), hl);
        float cdist = add_(h, hj);
        if (!(r2 < mul_(cdist, cdist))) continue;
        float ir = rsqrtf(r2);
        float r = mul_(r2, ir);
        V3f nh = scl(dd, ir);
        float Ej = voxel_E(A, j, mj);
        float kc = mul_(__fdividef(mul_(mul_(2.f, Ev), Ej), add_(Ev, Ej)), l);
        F = axpy(F, -mul_(kc, sub_(cdist, r)), nh);
        V3f vj = v3(jb.w, jc.x, jc.y);
        float cc = mul_(mul_(2.f, A.zc), fsqrt(mul_(fminf(d.m, dj.m), kc)));
        F = axpy(F, mul_(cc, dot3(sub(vj, s.v), nh)), nh);
      }
    }
  }
  if (A.floor_on) {
    float pen = sub_(h, add_(mt.z0, s.o.z));
    if (pen > 0.f) {
      float Fn = mul_(kv, pen);
      F.z = add_(F.z, fma_(-mul_(mul_(2.f, A.zc), fsqrt(mul_(d.m, kv))), s.v.z, Fn));
      float Fl2 = fma_(F.x, F.x, mul_(F.y, F.y));
      float vl2 = fma_(s.v.x, s.v.x, mul_(s.v.y, s.v.y));
      float mus = mul_(d.mu_s, Fn), mud = mul_(d.mu_k, Fn);
      float mus2 = mul_(mus, mus);
      bool zero_l = false;
      float fx = 0.f, fy = 0.f;  // unit direction of the dynamic friction force
      if (fl & 2u) {
        if (Fl2 <= mus2) zero_l = true;             // held by static friction
        else { fl &= ~2u; float i = rsqrtf(Fl2); fx = mul_(F.x, i); fy = mul_(F.y, i); }
      } else {
        float vth = mul_(mul_(mud, dt), d.inv_m);
        if (vl2 <= mul_(vth, vth) && Fl2 <= mus2) { zero_l = true; fl |= 2u; }  // halt
        else if (vl2 > 0.f) { float i = rsqrtf(vl2); fx = mul_(s.v.x, i); fy = mul_(s.v.y, i); }
        else { float i = rsqrtf(Fl2); fx = mul_(F.x, i); fy = mul_(F.y, i); }
      }
      if (zero_l) { F.x = 0.f; F.y = 0.f; s.v.x = 0.f; s.v.y = 0.f; }
      else { F.x = fma_(-mud, fx, F.x); F.y = fma_(-mud, fy, F.y); }
    } else {
      fl &= ~2u;
    }
  }
  // Sec 2.1.3: P += F dt, D += P/m dt; phi += M dt, theta += phi/I dt
  s.v = axpy(s.v, mul_(dt, d.inv_m), F);
  s.o = axpy(s.o, dt, s.v);
  s.w = axpy(s.w, mul_(dt, d.inv_I), M);
  s.q = integrate_rot(s.q, s.w, dt);
  float chk = s.o.x + s.o.y + s.o.z + s.v.x + s.v.y + s.v.z + s.w.x + s.w.y + s.w.z + s.q.w;
  if (!isfinite(chk)) record_bad(A, v);
  return fsqrt(fmaxf(dot3(s.v, s.v), 1e-30f));
}

// voxel_update, then the new state to st_out and changed flags in place.
__device__ __forceinline__ float voxel_finish(const StepArgs& A, int v, const VoxMeta& mt, VoxS s, V3f F, V3f M,
                                              float adT, float Ev, const DevMat* mats) {
  uint8_t fl;
  const float speed = voxel_update(A, v, mt, s, fl, F, M, adT, Ev, mats);
  store_vox(A.st_out, A.pitch, v, s);
  if (fl != mt.fl) A.flags[v] = fl;
  return speed;
}

// Collision horizon accumulator after a step (Sec 2.2.2, horizon reading):
// acc + 2 max|v| dt, the largest relative closure two voxels can make.
__device__ __forceinline__ float horizon_acc(float acc, float vmax, float dt) {
  return fma_(mul_(2.f, vmax), dt, acc);
}

// The horizon bookkeeping after a step, run by one CTA once every CTA's
// speeds are in: adds each body's closure to its accumulator (one
// accumulator with the largest speed of all bodies in a shared world), flags
// the bodies whose accumulator reached the threshold and zeroes the speeds.
// red: blockDim.x floats of shared scratch.
__device__ __forceinline__ void horizon_account(const StepArgs& A, float* red) {
  if (!A.h_world) {
    for (int b = threadIdx.x; b < A.n_bodies; b += blockDim.x) {
      const float vmax = __uint_as_float(atomicExch(&A.vmax_bits[b], 0u));
      float acc = horizon_acc(__ldcg(&A.h_acc[b]), vmax, A.dt_body[b]);
      if (acc >= A.h_threshold) {
        acc = 0.f;
        A.h_flag[b] = 1;
        atomicExch(A.h_any, 1);
      }
      A.h_acc[b] = acc;
    }
    return;
  }
  float m = 0.f;
  for (int b = threadIdx.x; b < A.n_bodies; b += blockDim.x)
    m = fmaxf(m, __uint_as_float(atomicExch(&A.vmax_bits[b], 0u)));
  red[threadIdx.x] = m;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  const float acc = horizon_acc(__ldcg(&A.h_acc[0]), red[0], A.dt_body[0]);
  const bool rebuild = acc >= A.h_threshold;
  if (rebuild)
    for (int b = threadIdx.x; b < A.n_bodies; b += blockDim.x) A.h_flag[b] = 1;
  if (threadIdx.x == 0) {
    A.h_acc[0] = rebuild ? 0.f : acc;
    if (rebuild) atomicExch(A.h_any, 1);
  }
}

// The horizon bookkeeping at the end of a step launch: each CTA, its tiles
// done, counts itself in; the last one runs horizon_account and zeroes the
// counter for the next launch.  red: blockDim.x floats of shared scratch.
__device__ __forceinline__ void horizon_tail(const StepArgs& A, float* red) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(A.h_done, 1u);
    reinterpret_cast<int*>(red)[0] = prev + 1 == gridDim.x;
  }
  __syncthreads();
  const bool last = reinterpret_cast<int*>(red)[0] != 0;
  __syncthreads();
  if (!last) return;
  __threadfence();
  horizon_account(A, red);
  if (threadIdx.x == 0) *A.h_done = 0u;
}

// Per-body max |v| for the collision horizon (max is order-independent).
__device__ __forceinline__ void horizon_max(const StepArgs& A, int b, bool active, float speed) {
  unsigned mask = __activemask();
  b = active ? b : 0;
  int b0 = __shfl_sync(mask, b, __ffs(mask) - 1);
  if (__all_sync(mask, b == b0 || !active)) {
    float s = active ? speed : 0.f;
    for (int o = 16; o > 0; o >>= 1) s = fmaxf(s, __shfl_xor_sync(mask, s, o));
    if ((threadIdx.x & 31) == __ffs(mask) - 1 && s > 0.f) atomicMax(&A.vmax_bits[b0], __float_as_uint(s));
  } else if (active && speed > 0.f) {
    atomicMax(&A.vmax_bits[b], __float_as_uint(speed));
  }
}

}  // namespace vx

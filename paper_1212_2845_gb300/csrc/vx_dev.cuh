// Device data layout and FP32 math of one explicit lattice step.
//
// State is structure-of-arrays: 13 float planes of `pitch` floats each
// (offset x,y,z from the lattice anchor, quaternion w,x,y,z, velocity x,y,z,
// angular velocity x,y,z), so every warp load or store of one component is
// one coalesced 128-byte transaction.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace vx {

enum Plane { OX = 0, OY, OZ, QW, QX, QY, QZ, VX, VY, VZ, WX, WY, WZ, NPLANE };

// Per-material constants precomputed on the host (mass and inertia depend on
// the lattice dimension l).
struct DevMat {
  float E;        // elastic modulus [Pa]
  float g_ratio;  // G / E = 1 / (2 (1 + nu))
  float cte;      // thermal expansion [1/K]
  float mu_s, mu_k;
  float m, inv_m; // rho l^3 and its inverse
  float I, inv_I; // m l^2 / 6 (solid cube) and its inverse
};

// Collision candidate capacity per surface voxel.
constexpr int kCandCap = 48;

// Status word bits.
constexpr int kStatusUnstable = 1;
constexpr int kStatusCapacity = 2;

struct StepArgs {
  int N;
  int64_t pitch;
  float l;
  float* st;               // NPLANE planes
  uint8_t* flags;          // bit 0 fixed, bit 1 static friction
  const uint8_t* mat;
  const uint32_t* lat;     // packed i | j << 11 | k << 22
  const int32_t* body;     // per voxel body index, or nullptr when single body
  const int32_t* nbr;      // 6 planes (-x,+x,-y,+y,-z,+z)
  const float* phase;      // per voxel or nullptr
  const float* logE;       // per voxel or nullptr
  const float* fext;       // 3 planes or nullptr
  const DevMat* mats;
  const float* dt_body;    // per body
  const float* origin;     // 3 per body
  float* bf;               // bond results: 9 components x 3 axes planes
  float zb, zg, zc, gz;
  int floor_on, collide_on;
  float actA, actT0;
  int64_t actP;
  int64_t step;
  // collisions
  const int32_t* sidx;     // per voxel: surface index or -1
  const int32_t* ccount;   // per surface voxel
  const int32_t* cand;     // per surface voxel, kCandCap slots
  unsigned* vmax_bits;     // per body, float bits of max |v|
  int* status;             // [0] bits, [1] first bad voxel, [2..3] step (int64)
};

// ---------------------------------------------------------------------------
// small vector / quaternion helpers (FP32)
// ---------------------------------------------------------------------------
struct V3f { float x, y, z; };
struct Qf { float w, x, y, z; };

__device__ __forceinline__ V3f v3(float a, float b, float c) { V3f r; r.x = a; r.y = b; r.z = c; return r; }
__device__ __forceinline__ V3f add(V3f a, V3f b) { return v3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ V3f sub(V3f a, V3f b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ V3f scl(V3f a, float s) { return v3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float dot3(V3f a, V3f b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3f cross3(V3f a, V3f b) {
  return v3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float comp(V3f a, int i) { return i == 0 ? a.x : (i == 1 ? a.y : a.z); }
// cyclic permutation taking lattice axis a to local x: local[i] = v[(i + a) % 3]
__device__ __forceinline__ V3f to_axis(V3f v, int a) {
  return a == 0 ? v : (a == 1 ? v3(v.y, v.z, v.x) : v3(v.z, v.x, v.y));
}
__device__ __forceinline__ V3f from_axis(V3f u, int a) {
  return a == 0 ? u : (a == 1 ? v3(u.z, u.x, u.y) : v3(u.y, u.z, u.x));
}

// Rotation matrix rows of unit quaternion q (body -> world).
struct M3f { V3f r0, r1, r2; };
__device__ __forceinline__ M3f qmat(Qf q) {
  float xx = q.x * q.x, yy = q.y * q.y, zz = q.z * q.z;
  float xy = q.x * q.y, xz = q.x * q.z, yz = q.y * q.z;
  float wx = q.w * q.x, wy = q.w * q.y, wz = q.w * q.z;
  M3f m;
  m.r0 = v3(1.f - 2.f * (yy + zz), 2.f * (xy - wz), 2.f * (xz + wy));
  m.r1 = v3(2.f * (xy + wz), 1.f - 2.f * (xx + zz), 2.f * (yz - wx));
  m.r2 = v3(2.f * (xz - wy), 2.f * (yz + wx), 1.f - 2.f * (xx + yy));
  return m;
}
// R v
__device__ __forceinline__ V3f mul(const M3f& m, V3f v) { return v3(dot3(m.r0, v), dot3(m.r1, v), dot3(m.r2, v)); }
// R^T v
__device__ __forceinline__ V3f mulT(const M3f& m, V3f v) {
  return v3(m.r0.x * v.x + m.r1.x * v.y + m.r2.x * v.z,
            m.r0.y * v.x + m.r1.y * v.y + m.r2.y * v.z,
            m.r0.z * v.x + m.r1.z * v.y + m.r2.z * v.z);
}
// (R^T e_a) - e_a: row a of R minus the unit vector, with the diagonal entry
// formed as -2 (sum of the other two squares) so no cancellation occurs.
__device__ __forceinline__ V3f row_dev(Qf q, int a) {
  if (a == 0) return v3(-2.f * (q.y * q.y + q.z * q.z), 2.f * (q.x * q.y - q.w * q.z), 2.f * (q.x * q.z + q.w * q.y));
  if (a == 1) return v3(2.f * (q.x * q.y + q.w * q.z), -2.f * (q.x * q.x + q.z * q.z), 2.f * (q.y * q.z - q.w * q.x));
  return v3(2.f * (q.x * q.z - q.w * q.y), 2.f * (q.y * q.z + q.w * q.x), -2.f * (q.x * q.x + q.y * q.y));
}

// Rotation vector of conj(q1) * q2 (shortest arc).
__device__ __forceinline__ V3f rel_rotvec(Qf a, Qf b) {
  float w = a.w * b.w + a.x * b.x + a.y * b.y + a.z * b.z;
  float x = a.w * b.x - a.x * b.w - a.y * b.z + a.z * b.y;
  float y = a.w * b.y + a.x * b.z - a.y * b.w - a.z * b.x;
  float z = a.w * b.z - a.x * b.y + a.y * b.x - a.z * b.w;
  if (w < 0.f) { w = -w; x = -x; y = -y; z = -z; }
  float s2 = x * x + y * y + z * z;
  float f;
  if (s2 < 1e-6f * w * w) {
    // 2 atan(t) / (t w) with t = s / w, Taylor series to t^4 (error < 2e-19)
    float t2 = s2 / (w * w);
    f = (2.f / w) * (1.f - t2 * (1.f / 3.f) + t2 * t2 * 0.2f);
  } else {
    float s = sqrtf(s2);
    f = 2.f * atan2f(s, w) / s;
  }
  return v3(x * f, y * f, z * f);
}

// q <- normalize(exp(w dt) * q)
__device__ __forceinline__ Qf integrate_rot(Qf q, V3f w, float dt) {
  float a2 = dot3(w, w) * dt * dt;
  float h2 = 0.25f * a2;  // (|w| dt / 2)^2
  float c, k;             // cos(|w|dt/2), sin(|w|dt/2)/|w|
  if (h2 < 1e-6f) {
    c = 1.f - 0.5f * h2 + h2 * h2 * (1.f / 24.f);
    k = 0.5f * dt * (1.f - h2 * (1.f / 6.f) + h2 * h2 * (1.f / 120.f));
  } else {
    float a = sqrtf(a2);
    float sn, cs;
    sincosf(0.5f * a, &sn, &cs);
    c = cs;
    k = sn * dt / a;
  }
  Qf d;
  d.w = c; d.x = w.x * k; d.y = w.y * k; d.z = w.z * k;
  Qf r;
  r.w = d.w * q.w - d.x * q.x - d.y * q.y - d.z * q.z;
  r.x = d.w * q.x + d.x * q.w + d.y * q.z - d.z * q.y;
  r.y = d.w * q.y - d.x * q.z + d.y * q.w + d.z * q.x;
  r.z = d.w * q.z + d.x * q.y - d.y * q.x + d.z * q.w;
  float n = 1.f / sqrtf(r.w * r.w + r.x * r.x + r.y * r.y + r.z * r.z);
  r.w *= n; r.x *= n; r.y *= n; r.z *= n;
  return r;
}

// Voxel state used by the bond computation.
struct VoxS { V3f o; Qf q; V3f v; V3f w; };

__device__ __forceinline__ VoxS load_vox(const float* __restrict__ st, int64_t pitch, int i) {
  VoxS s;
  s.o = v3(st[OX * pitch + i], st[OY * pitch + i], st[OZ * pitch + i]);
  s.q.w = st[QW * pitch + i]; s.q.x = st[QX * pitch + i]; s.q.y = st[QY * pitch + i]; s.q.z = st[QZ * pitch + i];
  s.v = v3(st[VX * pitch + i], st[VY * pitch + i], st[VZ * pitch + i]);
  s.w = v3(st[WX * pitch + i], st[WY * pitch + i], st[WZ * pitch + i]);
  return s;
}

// Temperature offset of a voxel at step n (Sec 2.3).
__device__ __forceinline__ float delta_T(const StepArgs& A, int v) {
  if (A.actP <= 0) return A.actT0;
  float frac = (float)(A.step % A.actP) / (float)A.actP;
  float ph = A.phase ? A.phase[v] : 0.f;
  return A.actT0 + A.actA * sinf(6.283185307179586f * frac + ph);
}

__device__ __forceinline__ float voxel_E(const StepArgs& A, int v, int m) {
  return A.logE ? expf(A.logE[v]) : A.mats[m].E;
}

// Result of one bond: force on voxel 1 (voxel 2 gets -F1), moments on both.
struct BondOut { V3f F1, M1, M2; };

// One bond along lattice axis a from voxel 1 (negative side) to voxel 2
// (Sec 2.1.2 co-rotational beam, Sec 2.1.5 damping, Sec 2.3 actuation).
__device__ __forceinline__ BondOut bond_eval(int a, const VoxS& s1, const VoxS& s2, float l,
                                             float E1, float E2, float G1, float G2,
                                             float mmin, float Imin, float eps, float zb) {
  float Ec = 2.f * E1 * E2 / (E1 + E2);
  float Gc = 2.f * G1 * G2 / (G1 + G2);
  float a1 = Ec * l;                       // E_c A / l
  float a2 = Gc * (l * l * l) * (1.f / 6.f);  // G_c J / l
  float b1 = a1;                           // 12 E_c I / l^3
  float b2 = Ec * (l * l) * 0.5f;          // 6 E_c I / l^2
  float b3 = Ec * (l * l * l) * (1.f / 6.f);  // 2 E_c I / l
  // position of voxel 2 in voxel 1's frame minus its rest vector l e_a:
  // R1^T (l e_a + do) - l e_a = R1^T do + l (R1^T e_a - e_a)
  M3f R1 = qmat(s1.q);
  V3f dO = sub(s2.o, s1.o);
  V3f p = add(mulT(R1, dO), scl(row_dev(s1.q, a), l));
  p = to_axis(p, a);
  float X = p.x - l * eps, Y = p.y, Z = p.z;
  V3f th = to_axis(rel_rotvec(s1.q, s2.q), a);
  // bond forces on the voxels (negated rows of [K] u, reduced form)
  V3f F1 = v3(a1 * X, b1 * Y - b2 * th.z, b1 * Z + b2 * th.y);
  V3f M1 = v3(a2 * th.x, -b2 * Z - b3 * th.y, b2 * Y - b3 * th.z);
  V3f M2 = v3(-a2 * th.x, -b2 * Z - 2.f * b3 * th.y, b2 * Y - 2.f * b3 * th.z);
  BondOut o;
  o.F1 = mul(R1, from_axis(F1, a));
  o.M1 = mul(R1, from_axis(M1, a));
  o.M2 = mul(R1, from_axis(M2, a));
  if (zb != 0.f) {
    // V_{2->1} = (v2 - Va) + (D2 - Da) x wa, with D2 - Da = (l e_a + do) / 2
    V3f wa = scl(add(s1.w, s2.w), 0.5f);
    V3f half = scl(dO, 0.5f);
    if (a == 0) half.x += 0.5f * l; else if (a == 1) half.y += 0.5f * l; else half.z += 0.5f * l;
    V3f V21 = add(scl(sub(s2.v, s1.v), 0.5f), cross3(half, wa));
    float c = 2.f * zb * sqrtf(mmin * a1);
    float cr = 2.f * zb * sqrtf(Imin * b3);
    o.F1 = add(o.F1, scl(V21, c));
    V3f dw = scl(sub(s2.w, s1.w), 0.5f * cr);   // cr (w2 - wa)
    o.M1 = add(o.M1, dw);
    o.M2 = sub(o.M2, dw);
  }
  return o;
}

}  // namespace vx

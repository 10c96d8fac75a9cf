// FP64 audit of the lattice state: linear and angular momentum, kinetic,
// elastic and gravitational energy (the only FP64 arithmetic on the GPU).
//
// Per voxel (Sec 2.1.3 state): P = m v, L = D x P + I w with D the absolute
// centre (lattice anchor + FP32 offset, formed in FP64), KE = |P|^2 / 2m +
// I |w|^2 / 2, U_g = -m g z.  Per bond (Sec 2.1.2): the elastic energy of the
// reduced beam, 1/2 u^T [K] u in the bond's co-rotational frame,
//   U = 1/2 (a1 X^2 + b1 Y^2 + b1 Z^2 + a2 tx^2 + 2 b3 ty^2 + 2 b3 tz^2)
//       - b2 Y tz + b2 Z ty,
// with X the axial stretch beyond the thermal rest length (Sec 2.3).
// Sums are deterministic: fixed per-thread order, a fixed shared-memory tree
// per block, then one block adding the block partials in index order.
#include "vx_dev.cuh"
#include "vx_kernels.h"

namespace vx {
namespace {

struct D3v { double x, y, z; };
__device__ __forceinline__ D3v d3(double a, double b, double c) { D3v r; r.x = a; r.y = b; r.z = c; return r; }
__device__ __forceinline__ D3v dsub(D3v a, D3v b) { return d3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ D3v dcross(D3v a, D3v b) {
  return d3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double ddot(D3v a, D3v b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// Absolute centre of voxel v in FP64.
__device__ __forceinline__ D3v centre(const AuditArgs& U, const StepArgs& A, int v, const VoxS& s) {
  const uint32_t p = A.lat[v];
  const int b = A.body ? A.body[v] : 0;
  const double l = U.l;
  return d3(U.origin[3 * b] + ((double)(int)(p & 2047u) + 0.5) * l + (double)s.o.x,
            U.origin[3 * b + 1] + ((double)(int)((p >> 11) & 2047u) + 0.5) * l + (double)s.o.y,
            U.origin[3 * b + 2] + ((double)(int)(p >> 22) + 0.5) * l + (double)s.o.z);
}

// R(q)^T d and the rotation vector of conj(q1) q2, in FP64.
__device__ __forceinline__ D3v rot_inv(Qf q, D3v d) {
  const double w = q.w, x = q.x, y = q.y, z = q.z;
  const double n = 1.0 / sqrt(w * w + x * x + y * y + z * z);
  const double qw = w * n, qx = x * n, qy = y * n, qz = z * n;
  // v' = v + 2 qv x (qv x v - qw v) for the conjugate rotation
  const D3v qv = d3(-qx, -qy, -qz);
  const D3v t = dcross(qv, d);
  const D3v t2 = d3(2.0 * t.x, 2.0 * t.y, 2.0 * t.z);
  const D3v c = dcross(qv, t2);
  return d3(d.x + qw * t2.x + c.x, d.y + qw * t2.y + c.y, d.z + qw * t2.z + c.z);
}
__device__ __forceinline__ D3v rel_rot(Qf a, Qf b) {
  const double aw = a.w, ax = a.x, ay = a.y, az = a.z, bw = b.w, bx = b.x, by = b.y, bz = b.z;
  double w = aw * bw + ax * bx + ay * by + az * bz;
  double x = aw * bx - ax * bw - ay * bz + az * by;
  double y = aw * by + ax * bz - ay * bw - az * bx;
  double z = aw * bz - ax * by + ay * bx - az * bw;
  if (w < 0.0) { w = -w; x = -x; y = -y; z = -z; }
  const double s = sqrt(x * x + y * y + z * z);
  const double f = s > 0.0 ? 2.0 * atan2(s, w) / s : 2.0 / w;
  return d3(x * f, y * f, z * f);
}

template <int a> __device__ __forceinline__ D3v to_ax(D3v v) {
  return a == 0 ? v : (a == 1 ? d3(v.y, v.z, v.x) : d3(v.z, v.x, v.y));
}

template <int a>
__device__ double bond_energy(const AuditArgs& U, const StepArgs& A, int v, int u, const VoxS& s1, const VoxS& s2) {
  const int m1 = A.mat[v], m2 = A.mat[u];
  const DevMat& d1 = A.mats[m1];
  const DevMat& d2 = A.mats[m2];
  const double E1 = A.logE ? exp((double)A.logE[v]) : U.E[m1];
  const double E2 = A.logE ? exp((double)A.logE[u]) : U.E[m2];
  const double G1 = E1 * U.g_ratio[m1], G2 = E2 * U.g_ratio[m2];
  const double Ec = 2.0 * E1 * E2 / (E1 + E2), Gc = 2.0 * G1 * G2 / (G1 + G2);
  const double l = U.l;
  const double a1 = Ec * l, a2 = Gc * l * l * l / 6.0, b1 = a1, b2 = Ec * l * l / 2.0, b3 = Ec * l * l * l / 6.0;
  const double eps = 0.5 * ((double)thermal_strain(A, v, d1) + (double)thermal_strain(A, u, d2));
  const D3v D1 = centre(U, A, v, s1), D2 = centre(U, A, u, s2);
  const D3v p = to_ax<a>(rot_inv(s1.q, dsub(D2, D1)));
  const D3v th = to_ax<a>(rel_rot(s1.q, s2.q));
  const double X = p.x - l * (1.0 + eps), Y = p.y, Z = p.z;
  return 0.5 * (a1 * X * X + b1 * Y * Y + b1 * Z * Z + a2 * th.x * th.x + 2.0 * b3 * th.y * th.y +
                2.0 * b3 * th.z * th.z) - b2 * Y * th.z + b2 * Z * th.y;
}

constexpr int kAudit = 10;  // P (3), L (3), KE linear, KE rotational, U elastic, U gravity

__global__ void __launch_bounds__(256) audit_blocks(StepArgs A, AuditArgs U, double* partial) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  double acc[kAudit];
#pragma unroll
  for (int k = 0; k < kAudit; ++k) acc[k] = 0.0;
  if (v < A.N) {
    const VoxS s = load_vox(A.st_in, A.pitch, v);
    const int m = A.mat[v];
    const double mass = U.mass[m], inertia = U.inertia[m];
    const D3v vel = d3(s.v.x, s.v.y, s.v.z), w = d3(s.w.x, s.w.y, s.w.z);
    const D3v P = d3(mass * vel.x, mass * vel.y, mass * vel.z);
    const D3v D = centre(U, A, v, s);
    const D3v L = dcross(D, P);
    acc[0] = P.x; acc[1] = P.y; acc[2] = P.z;
    acc[3] = L.x + inertia * w.x; acc[4] = L.y + inertia * w.y; acc[5] = L.z + inertia * w.z;
    acc[6] = 0.5 * mass * ddot(vel, vel);
    acc[7] = 0.5 * inertia * ddot(w, w);
    acc[9] = -mass * U.gz * D.z;
    const int up[3] = {A.nbr[(int64_t)1 * A.N + v], A.nbr[(int64_t)3 * A.N + v], A.nbr[(int64_t)5 * A.N + v]};
    if (up[0] >= 0) acc[8] += bond_energy<0>(U, A, v, up[0], s, load_vox(A.st_in, A.pitch, up[0]));
    if (up[1] >= 0) acc[8] += bond_energy<1>(U, A, v, up[1], s, load_vox(A.st_in, A.pitch, up[1]));
    if (up[2] >= 0) acc[8] += bond_energy<2>(U, A, v, up[2], s, load_vox(A.st_in, A.pitch, up[2]));
  }
  __shared__ double red[kAudit][256];
#pragma unroll
  for (int k = 0; k < kAudit; ++k) red[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o)
#pragma unroll
      for (int k = 0; k < kAudit; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x < kAudit) partial[(int64_t)blockIdx.x * kAudit + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void __launch_bounds__(256) audit_total(const double* partial, int nb, double* out) {
  __shared__ double red[kAudit][256];
  double acc[kAudit];
#pragma unroll
  for (int k = 0; k < kAudit; ++k) acc[k] = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < kAudit; ++k) acc[k] += partial[(int64_t)b * kAudit + k];
#pragma unroll
  for (int k = 0; k < kAudit; ++k) red[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o)
#pragma unroll
      for (int k = 0; k < kAudit; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x < kAudit) out[threadIdx.x] = red[threadIdx.x][0];
}

}  // namespace

int audit_partials(int N) { return (N + 255) / 256; }

void launch_audit(const StepArgs& A, const AuditArgs& U, double* partial, double* out, cudaStream_t s) {
  const int nb = audit_partials(A.N);
  audit_blocks<<<nb, 256, 0, s>>>(A, U, partial);
  audit_total<<<1, 256, 0, s>>>(partial, nb, out);
}

}  // namespace vx

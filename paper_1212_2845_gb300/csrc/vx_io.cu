// State transfer kernels: planar device state <-> interleaved caller layout.
#include "vx_kernels.h"

namespace vx {

// c: canonical index (caller layout), v: internal index (device planes)
__global__ void pack_state(const float* __restrict__ st, int64_t P, int N, const int32_t* __restrict__ iperm,
                           const uint8_t* __restrict__ flags, float* off, float* quat, float* vel, float* angvel,
                           uint8_t* fl) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  int64_t v = iperm[c];
  if (off) for (int a = 0; a < 3; ++a) off[3 * (int64_t)c + a] = st[state_index(OX + a, v, P)];
  if (quat) for (int a = 0; a < 4; ++a) quat[4 * (int64_t)c + a] = st[state_index(QW + a, v, P)];
  if (vel) for (int a = 0; a < 3; ++a) vel[3 * (int64_t)c + a] = st[state_index(VX + a, v, P)];
  if (angvel) for (int a = 0; a < 3; ++a) angvel[3 * (int64_t)c + a] = st[state_index(WX + a, v, P)];
  if (fl) fl[c] = flags[v];
}

__global__ void unpack_state(float* __restrict__ st, int64_t P, int N, const int32_t* __restrict__ iperm,
                             uint8_t* __restrict__ flags, const float* off, const float* quat, const float* vel,
                             const float* angvel, const uint8_t* fl) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  int64_t v = iperm[c];
  if (off) for (int a = 0; a < 3; ++a) st[state_index(OX + a, v, P)] = off[3 * (int64_t)c + a];
  if (quat) for (int a = 0; a < 4; ++a) st[state_index(QW + a, v, P)] = quat[4 * (int64_t)c + a];
  if (vel) for (int a = 0; a < 3; ++a) st[state_index(VX + a, v, P)] = vel[3 * (int64_t)c + a];
  if (angvel) for (int a = 0; a < 3; ++a) st[state_index(WX + a, v, P)] = angvel[3 * (int64_t)c + a];
  if (fl) flags[v] = fl[c];
}

__global__ void reset_state(float* __restrict__ st, int64_t P, int N, uint8_t* __restrict__ flags, float vx,
                            float vy, float vz) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= N) return;
  bool fixed = flags[v] & 1u;
  flags[v] &= 1u;  // keep fixed, clear static friction
  VoxS s;
  s.o = v3(0.f, 0.f, 0.f);
  s.q.w = 1.f; s.q.x = 0.f; s.q.y = 0.f; s.q.z = 0.f;
  s.v = fixed ? v3(0.f, 0.f, 0.f) : v3(vx, vy, vz);
  s.w = v3(0.f, 0.f, 0.f);
  store_vox(st, P, v, s);
}

// Linear velocity of every non-fixed voxel set to (vx, vy, vz); the rest of
// the state unchanged.
__global__ void set_velocity(float* __restrict__ st, int64_t P, int N, const uint8_t* __restrict__ flags, float vx,
                             float vy, float vz) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= N || (flags[v] & 1u)) return;
  VoxS s = load_vox(st, P, v);
  s.v = v3(vx, vy, vz);
  store_vox(st, P, v, s);
}

// Largest speed |v| over the voxels (the bits of a non-negative float order
// like unsigned integers, so an atomic max is exact and order-independent).
__global__ void max_speed(const float* __restrict__ st, int64_t P, int N, unsigned* __restrict__ out) {
  float m = 0.f;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < N; v += gridDim.x * blockDim.x) {
    const VoxS s = load_vox(st, P, v);
    m = fmaxf(m, sqrtf(s.v.x * s.v.x + s.v.y * s.v.y + s.v.z * s.v.z));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

void launch_max_speed(const float* st, int64_t pitch, int N, unsigned* out, cudaStream_t s) {
  const int nb = (N + 255) / 256 < 1024 ? (N + 255) / 256 : 1024;
  max_speed<<<nb, 256, 0, s>>>(st, pitch, N, out);
}

void launch_pack_state(const float* st, int64_t pitch, int N, const int32_t* iperm, const uint8_t* flags,
                       float* off, float* quat, float* vel, float* angvel, uint8_t* fl, cudaStream_t s) {
  pack_state<<<(N + 255) / 256, 256, 0, s>>>(st, pitch, N, iperm, flags, off, quat, vel, angvel, fl);
}

void launch_unpack_state(float* st, int64_t pitch, int N, const int32_t* iperm, uint8_t* flags, const float* off,
                         const float* quat, const float* vel, const float* angvel, const uint8_t* fl,
                         cudaStream_t s) {
  unpack_state<<<(N + 255) / 256, 256, 0, s>>>(st, pitch, N, iperm, flags, off, quat, vel, angvel, fl);
}

void launch_set_velocity(float* st, int64_t pitch, int N, const uint8_t* flags, float vx, float vy, float vz,
                         cudaStream_t s) {
  set_velocity<<<(N + 255) / 256, 256, 0, s>>>(st, pitch, N, flags, vx, vy, vz);
}

void launch_reset_state(float* st, int64_t pitch, int N, uint8_t* flags, float v0x, float v0y, float v0z,
                        cudaStream_t s) {
  reset_state<<<(N + 255) / 256, 256, 0, s>>>(st, pitch, N, flags, v0x, v0y, v0z);
}

}  // namespace vx

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
  if (off) for (int a = 0; a < 3; ++a) off[3 * (int64_t)c + a] = st[(OX + a) * P + v];
  if (quat) for (int a = 0; a < 4; ++a) quat[4 * (int64_t)c + a] = st[(QW + a) * P + v];
  if (vel) for (int a = 0; a < 3; ++a) vel[3 * (int64_t)c + a] = st[(VX + a) * P + v];
  if (angvel) for (int a = 0; a < 3; ++a) angvel[3 * (int64_t)c + a] = st[(WX + a) * P + v];
  if (fl) fl[c] = flags[v];
}

__global__ void unpack_state(float* __restrict__ st, int64_t P, int N, const int32_t* __restrict__ iperm,
                             uint8_t* __restrict__ flags, const float* off, const float* quat, const float* vel,
                             const float* angvel, const uint8_t* fl) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  int64_t v = iperm[c];
  if (off) for (int a = 0; a < 3; ++a) st[(OX + a) * P + v] = off[3 * (int64_t)c + a];
  if (quat) for (int a = 0; a < 4; ++a) st[(QW + a) * P + v] = quat[4 * (int64_t)c + a];
  if (vel) for (int a = 0; a < 3; ++a) st[(VX + a) * P + v] = vel[3 * (int64_t)c + a];
  if (angvel) for (int a = 0; a < 3; ++a) st[(WX + a) * P + v] = angvel[3 * (int64_t)c + a];
  if (fl) flags[v] = fl[c];
}

__global__ void reset_state(float* __restrict__ st, int64_t P, int N, uint8_t* __restrict__ flags, float vx,
                            float vy, float vz) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= N) return;
  bool fixed = flags[v] & 1u;
  flags[v] &= 1u;  // keep fixed, clear static friction
  st[OX * P + v] = 0.f; st[OY * P + v] = 0.f; st[OZ * P + v] = 0.f;
  st[QW * P + v] = 1.f; st[QX * P + v] = 0.f; st[QY * P + v] = 0.f; st[QZ * P + v] = 0.f;
  st[VX * P + v] = fixed ? 0.f : vx; st[VY * P + v] = fixed ? 0.f : vy; st[VZ * P + v] = fixed ? 0.f : vz;
  st[WX * P + v] = 0.f; st[WY * P + v] = 0.f; st[WZ * P + v] = 0.f;
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

void launch_reset_state(float* st, int64_t pitch, int N, uint8_t* flags, float v0x, float v0y, float v0z,
                        cudaStream_t s) {
  reset_state<<<(N + 255) / 256, 256, 0, s>>>(st, pitch, N, flags, v0x, v0y, v0z);
}

}  // namespace vx

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

// Runs over the internal order (perm: internal -> canonical), so that the
// state planes are written in runs and the caller's arrays are the ones read
// out of order.  With dmax set (collisions on), the largest distance between
// a voxel's written and current offsets is recorded per body (float bits,
// atomicMax: the maximum does not depend on the order): one atomic per CTA
// when all its voxels belong to one body (bodies are contiguous in the
// internal order), else per voxel.
__global__ void __launch_bounds__(256) unpack_state(float* __restrict__ st, int64_t P, int N,
                                                    const int32_t* __restrict__ perm, uint8_t* __restrict__ flags,
                                                    const float* off, const float* quat, const float* vel,
                                                    const float* angvel, const uint8_t* fl, const int32_t* body,
                                                    unsigned* dmax) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = v < N;
  float d2 = 0.f;
  int b = 0;
  if (active) {
    const int64_t c = perm[v];
    if (off)
      for (int a = 0; a < 3; ++a) {
        const float o1 = off[3 * c + a];
        if (dmax) {
          const float dd = __fsub_rn(o1, st[state_index(OX + a, v, P)]);
          d2 = __fmaf_rn(dd, dd, d2);
        }
        st[state_index(OX + a, v, P)] = o1;
      }
    if (quat) for (int a = 0; a < 4; ++a) st[state_index(QW + a, v, P)] = quat[4 * c + a];
    if (vel) for (int a = 0; a < 3; ++a) st[state_index(VX + a, v, P)] = vel[3 * c + a];
    if (angvel) for (int a = 0; a < 3; ++a) st[state_index(WX + a, v, P)] = angvel[3 * c + a];
    if (fl) flags[v] = fl[c];
    if (body) b = body[v];
  }
  if (!dmax || !off) return;  // uniform over the grid
  const float d = sqrtf(d2);
  const int b_first = body ? body[blockIdx.x * blockDim.x] : 0;  // the CTA's first voxel exists
  float m = d;
  if (__syncthreads_and(!active || b == b_first)) {
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ float red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
      if (m > 0.f) atomicMax(&dmax[b_first], __float_as_uint(m));
    }
  } else if (active && d > 0.f) {
    atomicMax(&dmax[b], __float_as_uint(d));
  }
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

void launch_unpack_state(float* st, int64_t pitch, int N, const int32_t* perm, uint8_t* flags, const float* off,
                         const float* quat, const float* vel, const float* angvel, const uint8_t* fl,
                         cudaStream_t s, const int32_t* body, unsigned* dmax) {
  if (N > 0)
    unpack_state<<<(N + 255) / 256, 256, 0, s>>>(st, pitch, N, perm, flags, off, quat, vel, angvel, fl, body, dmax);
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

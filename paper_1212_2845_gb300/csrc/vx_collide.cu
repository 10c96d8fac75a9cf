// Collision candidates between surface voxels (Sec 2.2.2).
//
// A pair (i, j) of surface voxels of one body is a candidate when their
// lattice Manhattan distance exceeds 3 and their centres are closer than the
// 2-voxel collision horizon.  In a shared world (bodies collide with each
// other) voxels of different bodies pair on distance alone, and every body's
// quantised origin rint(origin 2^K) puts all bodies in one integer frame.  The distance test runs on integers: each
// coordinate is anchor * Q + rint(offset * 2^K) (2^K ~ 65536 / l, exact power
// of two scaling of the FP32 offset), so the candidate set is a bit-exact
// function of the FP32 state.
//
// Rebuild pipeline (all on the stream, no host round trip):
//   horizon_update  accumulates 2 max|v| dt per body and raises a body's
//                   rebuild flag at the threshold (in a shared world of
//                   several bodies, one accumulator for all of them)
//   rebuild_all     one cooperative launch whose phases are separated by
//                   grid barriers; it returns at once when no body is flagged
//                   (the usual step), otherwise:
//     quantise      integer coordinates, cell (edge = horizon) and hash
//                   bucket of every surface voxel; counts per bucket
//     scan          exclusive prefix sum of the bucket counts (per-CTA chunk
//                   scans, then chunk offsets)
//     scatter       surface voxels grouped by bucket (order within a bucket
//                   is irrelevant: lists are sorted below)
//     query         27 neighbour cells per surface voxel of a flagged body;
//                   candidates sorted ascending by canonical index
//     finish        clears flags, counts the rebuild
#include "vx_collide.cuh"

#include <algorithm>

namespace vx {

// Shared world: one accumulator over all bodies (relative motion between
// bodies counts), kept in slot 0; a rebuild flags every body.  One block.
__global__ void horizon_update_world(CollideArgs C) {
  __shared__ float red[256];
  float m = 0.f;
  for (int b = threadIdx.x; b < C.n_bodies; b += blockDim.x) {
    m = fmaxf(m, __uint_as_float(C.vmax_bits[b]));
    C.vmax_bits[b] = 0u;
  }
  red[threadIdx.x] = m;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  const float acc = horizon_acc(C.acc[0], red[0], C.dt_body[0]);
  const bool rebuild = acc >= C.threshold;
  __syncthreads();
  if (rebuild)
    for (int b = threadIdx.x; b < C.n_bodies; b += blockDim.x) C.flag[b] = 1;
  if (threadIdx.x == 0) {
    C.acc[0] = rebuild ? 0.f : acc;
    if (rebuild) atomicExch(C.any, 1);
  }
}

__global__ void horizon_update(CollideArgs C) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= C.n_bodies) return;
  float vmax = __uint_as_float(C.vmax_bits[b]);
  C.vmax_bits[b] = 0u;
  float acc = horizon_acc(C.acc[b], vmax, C.dt_body[b]);
  if (acc >= C.threshold) {
    acc = 0.f;
    C.flag[b] = 1;
    atomicExch(C.any, 1);
  }
  C.acc[b] = acc;
}

constexpr int kRebuildThreads = 256;

// The whole rebuild in one cooperative launch (all CTAs co-resident; phases
// separated by grid barriers, whose waits are bounded: on a timeout the
// launch ends with the timeout status bit set).  Five CTAs per SM (at most 48
// registers) give 194,560 threads, one per searched voxel of a 192,848-voxel
// ball surface in a single pass of the query; at four the query needs two.
__global__ void __launch_bounds__(kRebuildThreads, 5) rebuild_all(CollideArgs C) {
  extern __shared__ int ws[];  // kWarpWs ints per warp
  if (*C.any == 0) return;  // the same value for every CTA: set by an earlier launch
  rebuild_phases(C, gridDim.x + C.extra, ws);
}

// The largest written displacement d of a body moves any two of its voxels
// relative to each other by at most 2 d, as a step's 2 max|v| dt does; the
// relative margin 2^-16 covers the rounding of d.  One block.
__global__ void write_horizon(CollideArgs C, unsigned* dmax, int world) {
  __shared__ float red[256];
  const bool all = (C.status[0] & (kStatusTimeout | kStatusCapacity)) != 0;
  float m = 0.f;
  for (int b = threadIdx.x; b < C.n_bodies; b += blockDim.x) {
    const float d = __uint_as_float(dmax[b]);
    dmax[b] = 0u;
    if (world) {
      m = fmaxf(m, d);
    } else {
      float acc = __fmaf_rn(2.f * d, 1.f + 0x1p-16f, C.acc[b]);
      if (all || acc >= C.threshold) {
        acc = 0.f;
        C.flag[b] = 1;
        atomicExch(C.any, 1);
      }
      C.acc[b] = acc;
    }
  }
  if (!world) return;  // uniform
  red[threadIdx.x] = m;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  const float acc = __fmaf_rn(2.f * red[0], 1.f + 0x1p-16f, C.acc[0]);
  const bool rebuild = all || acc >= C.threshold;
  if (rebuild)
    for (int b = threadIdx.x; b < C.n_bodies; b += blockDim.x) C.flag[b] = 1;
  if (threadIdx.x == 0) {
    C.acc[0] = rebuild ? 0.f : acc;
    if (rebuild) atomicExch(C.any, 1);
  }
}

void launch_write_horizon(const CollideArgs& C, unsigned* dmax, int world, cudaStream_t st) {
  write_horizon<<<1, 256, 0, st>>>(C, dmax, world);
}

// Raise every body's rebuild flag (forced rebuild).
__global__ void flag_all(CollideArgs C) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < C.n_bodies; b += gridDim.x * blockDim.x) {
    C.flag[b] = 1;
    C.acc[b] = 0.f;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *C.any = 1;
}

int rebuild_grid_limit() {
  static int cached[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  if (!cached[dev]) {
    int per_sm = 0, n_sm = 0;
    const size_t ws = (size_t)(kRebuildThreads / 32) * kWarpWs * sizeof(int);
    if (cudaFuncSetAttribute((const void*)rebuild_all, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ws) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rebuild_all, kRebuildThreads, ws) != cudaSuccess ||
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || per_sm < 1)
      return 0;
    cached[dev] = per_sm * n_sm;
  }
  return cached[dev];
}

void launch_rebuild(const CollideArgs& C, cudaStream_t st) {
  if (C.S == 0) return;
  const int limit = rebuild_grid_limit();
  // one warp per searched voxel in the query, one thread per bucket in the scan
  const int warps_per_cta = kRebuildThreads / 32;
  const int want = std::max((C.S + warps_per_cta - 1) / warps_per_cta, (C.H + kRebuildThreads - 1) / kRebuildThreads);
  int grid = std::min(std::min(want, limit), kRebuildMaxGrid);
  if (grid < 1) grid = 1;
  void* args[1] = {const_cast<CollideArgs*>(&C)};
  const size_t ws = (size_t)(kRebuildThreads / 32) * kWarpWs * sizeof(int);
  cudaLaunchCooperativeKernel((const void*)rebuild_all, dim3(grid), dim3(kRebuildThreads), args, ws, st);
}

void launch_flag_all(const CollideArgs& C, cudaStream_t st) {
  flag_all<<<1, 256, 0, st>>>(C);
}

void launch_horizon(const CollideArgs& C, cudaStream_t st) {
  if (C.qorg) {
    horizon_update_world<<<1, 256, 0, st>>>(C);
    return;
  }
  horizon_update<<<(C.n_bodies + 255) / 256, 256, 0, st>>>(C);
}

}  // namespace vx

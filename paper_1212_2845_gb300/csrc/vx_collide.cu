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
#include "vx_dev.cuh"
#include "vx_kernels.h"

#include <algorithm>

namespace vx {

__device__ __forceinline__ int64_t floordiv(int64_t a, int64_t b) {
  int64_t q = a / b;
  return (a % b != 0 && ((a < 0) != (b < 0))) ? q - 1 : q;
}

__device__ __forceinline__ uint32_t cell_hash(int64_t cx, int64_t cy, int64_t cz, uint32_t mask) {
  uint64_t h = (uint64_t)cx * 0x9E3779B97F4A7C15ull ^ (uint64_t)cy * 0xC2B2AE3D27D4EB4Full ^
               (uint64_t)cz * 0x165667B19E3779F9ull;
  h ^= h >> 29;
  return (uint32_t)h & mask;
}

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

__device__ __forceinline__ void quantise_one(const CollideArgs& C, int s) {
  int v = C.surf[s];
  uint32_t lp = C.lat[v];
  int64_t ijk[3] = {(int64_t)(lp & 2047u), (int64_t)((lp >> 11) & 2047u), (int64_t)(lp >> 22)};
  const int64_t* qo = C.qorg ? C.qorg + 3 * (C.body ? C.body[v] : 0) : nullptr;
  int64_t xq[3];
  for (int a = 0; a < 3; ++a) {
    float o = C.st[(int64_t)v * C.ostride_v + a * C.ostride_a];
    xq[a] = (qo ? qo[a] : 0) + ijk[a] * C.Q + llrintf(ldexpf(o, C.K));
    C.xq[(int64_t)a * C.S + s] = xq[a];
  }
  int64_t cs = 2 * C.Q;
  const int64_t cx = floordiv(xq[0], cs), cy = floordiv(xq[1], cs), cz = floordiv(xq[2], cs);
  C.cell[s] = make_int4((int)cx, (int)cy, (int)cz, 0);  // cells of a world fit in 32 bits
  uint32_t h = cell_hash(cx, cy, cz, C.H - 1);
  C.bucket[s] = h;
  atomicAdd(&C.hcount[h], 1u);
}

// Exclusive scan of x over the CTA (all threads call it); returns this
// thread's prefix and the CTA total.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t* warp_tot, uint32_t* block_total) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t inc = x;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) warp_tot[w] = inc;
  __syncthreads();
  if (w == 0) {
    uint32_t t = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0u;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    warp_tot[lane] = t;
  }
  __syncthreads();
  uint32_t pre = (w > 0 ? warp_tot[w - 1] : 0u) + inc - x;
  *block_total = warp_tot[(blockDim.x >> 5) - 1];
  __syncthreads();
  return pre;
}

__device__ __forceinline__ void query_one(const CollideArgs& C, int s) {
  int v = C.surf[s];
  int b = C.body ? C.body[v] : 0;
  if (!C.flag[b]) return;
  int64_t x0 = C.xq[s], y0 = C.xq[(int64_t)C.S + s], z0 = C.xq[2 * (int64_t)C.S + s];
  int64_t cs = 2 * C.Q;
  const int4 c0 = C.cell[s];
  const int cx = c0.x, cy = c0.y, cz = c0.z;
  uint32_t lp = C.lat[v];
  int vi = (int)(lp & 2047u), vj = (int)((lp >> 11) & 2047u), vk = (int)(lp >> 22);
  int64_t r2max = cs * cs;  // (2 Q)^2
  int list[kCandCap];
  int n = 0;
  bool overflow = false;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const int ncx = cx + dx, ncy = cy + dy, ncz = cz + dz;
        uint32_t h = cell_hash(ncx, ncy, ncz, C.H - 1);
        uint32_t e0 = C.hstart[h], e1 = C.hstart[h + 1];
        for (uint32_t e = e0; e < e1; ++e) {
          int t = C.sorted[e];
          if (t == s) continue;
          const int4 c1 = C.cell[t];
          if (c1.x != ncx || c1.y != ncy || c1.z != ncz) continue;  // another cell in the same bucket
          int64_t x1 = C.xq[t], y1 = C.xq[(int64_t)C.S + t], z1 = C.xq[2 * (int64_t)C.S + t];
          int u = C.surf[t];
          if (C.body && C.body[u] != b) {
            if (!C.qorg) continue;  // bodies are separate worlds
          } else {
            uint32_t lq = C.lat[u];
            int man = abs((int)(lq & 2047u) - vi) + abs((int)((lq >> 11) & 2047u) - vj) + abs((int)(lq >> 22) - vk);
            if (man <= 3) continue;
          }
          int64_t ddx = x1 - x0, ddy = y1 - y0, ddz = z1 - z0;
          if (ddx * ddx + ddy * ddy + ddz * ddz >= r2max) continue;
          if (n < kCandCap) list[n++] = u; else overflow = true;
        }
      }
  // insertion sort ascending (lists are short)
  for (int i = 1; i < n; ++i) {
    int x = list[i];
    int k = i - 1;
    while (k >= 0 && list[k] > x) { list[k + 1] = list[k]; --k; }
    list[k + 1] = x;
  }
  int32_t* out = C.cand + (int64_t)s * kCandCap;
  for (int i = 0; i < n; ++i) out[i] = list[i];
  C.ccount[s] = n;
  if (overflow) atomicOr(C.status, kStatusCapacity);
}

constexpr int kRebuildThreads = 256;

// The whole rebuild in one cooperative launch (all CTAs co-resident; phases
// separated by grid barriers, whose waits are bounded: on a timeout the
// launch ends with the timeout status bit set).
__global__ void __launch_bounds__(kRebuildThreads) rebuild_all(CollideArgs C) {
  __shared__ uint32_t warp_tot[32];
  __shared__ uint32_t offset;
  if (*C.any == 0) return;  // the same value for every CTA: set by an earlier launch
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
  const unsigned G = gridDim.x;
  // zero the bucket counters
  for (int i = tid; i < C.H; i += nthr) { C.hcount[i] = 0u; C.hcursor[i] = 0u; }
  if (!grid_barrier(C.bar, G, C.spins, C.status)) return;
  for (int s = tid; s < C.S; s += nthr) quantise_one(C, s);
  if (!grid_barrier(C.bar, G, C.spins, C.status)) return;
  // scan: CTA c owns buckets [c chunk, (c + 1) chunk)
  const int chunk = (C.H + (int)G - 1) / (int)G;
  const int b0 = min(C.H, (int)blockIdx.x * chunk), b1 = min(C.H, b0 + chunk);
  uint32_t carry = 0u;
  for (int base = b0; base < b1; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const uint32_t x = i < b1 ? C.hcount[i] : 0u;
    uint32_t tot;
    const uint32_t pre = block_exclusive_scan(x, warp_tot, &tot);
    if (i < b1) C.hstart[i] = carry + pre;
    carry += tot;
  }
  if (threadIdx.x == 0) C.bsum[blockIdx.x] = carry;
  if (!grid_barrier(C.bar, G, C.spins, C.status)) return;
  {
    // offset of this CTA's chunk: sum of the chunk totals before it (fixed order)
    uint32_t part = 0u;
    for (int c = threadIdx.x; c < (int)blockIdx.x; c += blockDim.x) part += C.bsum[c];
    uint32_t tot;
    block_exclusive_scan(part, warp_tot, &tot);
    if (threadIdx.x == 0) offset = tot;
    __syncthreads();
    for (int i = b0 + threadIdx.x; i < b1; i += blockDim.x) C.hstart[i] += offset;
    if (blockIdx.x == G - 1 && threadIdx.x == 0) C.hstart[C.H] = offset + carry;
  }
  if (!grid_barrier(C.bar, G, C.spins, C.status)) return;
  for (int s = tid; s < C.S; s += nthr) {
    const uint32_t h = C.bucket[s];
    C.sorted[C.hstart[h] + atomicAdd(&C.hcursor[h], 1u)] = s;
  }
  if (!grid_barrier(C.bar, G, C.spins, C.status)) return;
  for (int s = tid; s < C.S; s += nthr) query_one(C, s);
  if (!grid_barrier(C.bar, G, C.spins, C.status)) return;
  if (blockIdx.x == 0) {
    for (int b = threadIdx.x; b < C.n_bodies; b += blockDim.x) C.flag[b] = 0;
    __syncthreads();
    if (threadIdx.x == 0) { *C.any = 0; *C.n_rebuilds += 1; }
  }
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
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rebuild_all, kRebuildThreads, 0) != cudaSuccess ||
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || per_sm < 1)
      return 0;
    cached[dev] = per_sm * n_sm;
  }
  return cached[dev];
}

void launch_rebuild(const CollideArgs& C, cudaStream_t st) {
  if (C.S == 0) return;
  const int limit = rebuild_grid_limit();
  const int want = (std::max(C.S, C.H) + kRebuildThreads - 1) / kRebuildThreads;
  int grid = std::min(std::min(want, limit), kRebuildMaxGrid);
  if (grid < 1) grid = 1;
  void* args[1] = {const_cast<CollideArgs*>(&C)};
  cudaLaunchCooperativeKernel((const void*)rebuild_all, dim3(grid), dim3(kRebuildThreads), args, 0, st);
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

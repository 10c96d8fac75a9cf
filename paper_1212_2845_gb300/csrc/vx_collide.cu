// Collision candidates between surface voxels (Sec 2.2.2).
//
// A pair (i, j) of surface voxels of one body is a candidate when their
// lattice Manhattan distance exceeds 3 and their centres are closer than the
// 2-voxel collision horizon.  The distance test runs on integers: each
// coordinate is anchor * Q + rint(offset * 2^K) (2^K ~ 65536 / l, exact power
// of two scaling of the FP32 offset), so the candidate set is a bit-exact
// function of the FP32 state.
//
// Rebuild pipeline (all on the stream, no host round trip):
//   horizon_update  accumulates 2 max|v| dt per body and raises a body's
//                   rebuild flag at the threshold
//   quantise        integer coordinates, cell (edge = horizon) and hash bucket
//                   of every surface voxel; counts per bucket
//   scan            exclusive prefix sum of the bucket counts
//   scatter         surface voxels grouped by bucket (order within a bucket
//                   is irrelevant: lists are sorted below)
//   query           27 neighbour cells per surface voxel of a flagged body;
//                   candidates sorted ascending by canonical index
//   finish          clears flags, counts the rebuild
// Every kernel returns at once when no body is flagged.
#include "vx_dev.cuh"
#include "vx_kernels.h"

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

__global__ void horizon_update(CollideArgs C) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= C.n_bodies) return;
  float vmax = __uint_as_float(C.vmax_bits[b]);
  C.vmax_bits[b] = 0u;
  float acc = C.acc[b] + 2.f * vmax * C.dt_body[b];
  if (acc >= C.threshold) {
    acc = 0.f;
    C.flag[b] = 1;
    atomicExch(C.any, 1);
  }
  C.acc[b] = acc;
}

__global__ void quantise(CollideArgs C) {
  if (*C.any == 0) return;
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= C.S) return;
  int v = C.surf[s];
  uint32_t lp = C.lat[v];
  int64_t ijk[3] = {(int64_t)(lp & 2047u), (int64_t)((lp >> 11) & 2047u), (int64_t)(lp >> 22)};
  int64_t xq[3];
  for (int a = 0; a < 3; ++a) {
    float o = C.st[(int64_t)v * C.ostride_v + a * C.ostride_a];
    xq[a] = ijk[a] * C.Q + llrintf(ldexpf(o, C.K));
    C.xq[(int64_t)a * C.S + s] = xq[a];
  }
  int64_t cs = 2 * C.Q;
  uint32_t h = cell_hash(floordiv(xq[0], cs), floordiv(xq[1], cs), floordiv(xq[2], cs), C.H - 1);
  C.bucket[s] = h;
  atomicAdd(&C.hcount[h], 1u);
}

__global__ void zero_counts(CollideArgs C) {
  if (*C.any == 0) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < C.H; i += gridDim.x * blockDim.x) {
    C.hcount[i] = 0u;
    C.hcursor[i] = 0u;
  }
}

// Exclusive scan of hcount[0..H) into hstart[0..H] in three phases:
// per-block scan, scan of the block sums (one block), add the block offsets.
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

__global__ void __launch_bounds__(1024) scan_blocks(CollideArgs C) {
  if (*C.any == 0) return;
  __shared__ uint32_t warp_tot[32];
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t x = i < C.H ? C.hcount[i] : 0u;
  uint32_t tot;
  uint32_t pre = block_exclusive_scan(x, warp_tot, &tot);
  if (i < C.H) C.hstart[i] = pre;
  if (threadIdx.x == 0) C.bsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) scan_sums(CollideArgs C, int nb) {
  if (*C.any == 0) return;
  __shared__ uint32_t warp_tot[32];
  uint32_t carry = 0u;
  for (int base = 0; base < nb; base += blockDim.x) {
    int i = base + threadIdx.x;
    uint32_t x = i < nb ? C.bsum[i] : 0u;
    uint32_t tot;
    uint32_t pre = block_exclusive_scan(x, warp_tot, &tot);
    if (i < nb) C.bsum[i] = carry + pre;
    carry += tot;
  }
  if (threadIdx.x == 0) C.hstart[C.H] = carry;
}

__global__ void __launch_bounds__(1024) scan_add(CollideArgs C) {
  if (*C.any == 0) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < C.H) C.hstart[i] += C.bsum[blockIdx.x];
}

__global__ void scatter(CollideArgs C) {
  if (*C.any == 0) return;
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= C.S) return;
  uint32_t h = C.bucket[s];
  uint32_t pos = C.hstart[h] + atomicAdd(&C.hcursor[h], 1u);
  C.sorted[pos] = s;
}

__global__ void query(CollideArgs C) {
  if (*C.any == 0) return;
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= C.S) return;
  int v = C.surf[s];
  int b = C.body ? C.body[v] : 0;
  if (!C.flag[b]) return;
  int64_t x0 = C.xq[s], y0 = C.xq[(int64_t)C.S + s], z0 = C.xq[2 * (int64_t)C.S + s];
  int64_t cs = 2 * C.Q;
  int64_t cx = floordiv(x0, cs), cy = floordiv(y0, cs), cz = floordiv(z0, cs);
  uint32_t lp = C.lat[v];
  int vi = (int)(lp & 2047u), vj = (int)((lp >> 11) & 2047u), vk = (int)(lp >> 22);
  int64_t r2max = cs * cs;  // (2 Q)^2
  int list[kCandCap];
  int n = 0;
  bool overflow = false;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        int64_t ncx = cx + dx, ncy = cy + dy, ncz = cz + dz;
        uint32_t h = cell_hash(ncx, ncy, ncz, C.H - 1);
        uint32_t e0 = C.hstart[h], e1 = C.hstart[h + 1];
        for (uint32_t e = e0; e < e1; ++e) {
          int t = C.sorted[e];
          if (t == s) continue;
          int64_t x1 = C.xq[t], y1 = C.xq[(int64_t)C.S + t], z1 = C.xq[2 * (int64_t)C.S + t];
          if (floordiv(x1, cs) != ncx || floordiv(y1, cs) != ncy || floordiv(z1, cs) != ncz) continue;
          int u = C.surf[t];
          if (C.body && C.body[u] != b) continue;
          uint32_t lq = C.lat[u];
          int man = abs((int)(lq & 2047u) - vi) + abs((int)((lq >> 11) & 2047u) - vj) + abs((int)(lq >> 22) - vk);
          if (man <= 3) continue;
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

__global__ void finish(CollideArgs C) {
  // one block: every thread must see the same *any before it is cleared
  if (*C.any == 0) return;
  for (int b = threadIdx.x; b < C.n_bodies; b += blockDim.x) C.flag[b] = 0;
  __syncthreads();
  if (threadIdx.x == 0) { *C.any = 0; *C.n_rebuilds += 1; }
}

// Raise every body's rebuild flag (forced rebuild).
__global__ void flag_all(CollideArgs C) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < C.n_bodies; b += gridDim.x * blockDim.x) {
    C.flag[b] = 1;
    C.acc[b] = 0.f;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *C.any = 1;
}

void launch_rebuild(const CollideArgs& C, cudaStream_t st) {
  int S = C.S;
  if (S == 0) return;
  int tb = 256;
  int nb = (C.H + 1023) / 1024;
  zero_counts<<<nb, 1024, 0, st>>>(C);
  quantise<<<(S + tb - 1) / tb, tb, 0, st>>>(C);
  scan_blocks<<<nb, 1024, 0, st>>>(C);
  scan_sums<<<1, 1024, 0, st>>>(C, nb);
  scan_add<<<nb, 1024, 0, st>>>(C);
  scatter<<<(S + tb - 1) / tb, tb, 0, st>>>(C);
  query<<<(S + 127) / 128, 128, 0, st>>>(C);
  finish<<<1, 256, 0, st>>>(C);
}

void launch_flag_all(const CollideArgs& C, cudaStream_t st) {
  flag_all<<<1, 256, 0, st>>>(C);
}

void launch_horizon(const CollideArgs& C, cudaStream_t st) {
  horizon_update<<<(C.n_bodies + 255) / 256, 256, 0, st>>>(C);
}

}  // namespace vx

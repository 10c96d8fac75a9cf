// Device side of the collision-candidate rebuild (Sec 2.2.2), shared by the
// rebuild launch and the multi-step launch that rebuilds between its steps.
// See vx_collide.cu for the pipeline.
#pragma once
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
  if (VX_IN_BOUNDS(C.status, h, C.H, kSiteBucket)) atomicAdd(&C.hcount[h], 1u);
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

// Candidates of searched voxel s, found by one thread (27 neighbour cells in
// a row): the query when there are many more searched voxels than warps.
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
  for (int dz = -1; dz <= 1; ++dz) {
    for (int q = 0; q < 9; ++q) {
        const int ncx = cx + q % 3 - 1, ncy = cy + q / 3 - 1, ncz = cz + dz;
        const uint32_t hq = cell_hash(ncx, ncy, ncz, C.H - 1);
        const uint32_t e0 = C.hstart[hq], e1 = C.hstart[hq + 1];
        auto take = [&](uint32_t e, int4 c1, int4 f) {
          if (c1.w == s) return;
          if (c1.x != ncx || c1.y != ncy || c1.z != ncz) return;  // another cell in the same bucket
          const int u = f.x;
          if (C.body && f.z != b) {
            if (!C.qorg) return;  // bodies are separate worlds
          } else {
            const uint32_t lq = (uint32_t)f.y;
            int man = abs((int)(lq & 2047u) - vi) + abs((int)((lq >> 11) & 2047u) - vj) + abs((int)(lq >> 22) - vk);
            if (man <= 3) return;
          }
          const int64_t x1 = C.sxq[e], y1 = C.sxq[(int64_t)C.S + e], z1 = C.sxq[2 * (int64_t)C.S + e];
          int64_t ddx = x1 - x0, ddy = y1 - y0, ddz = z1 - z0;
          if (ddx * ddx + ddy * ddy + ddz * ddz >= r2max) return;
          if (n < kCandCap) list[n++] = u; else overflow = true;
        };
        // two entries requested at once: their loads overlap
        for (uint32_t e = e0; e < e1; e += 2) {
          if (!VX_IN_BOUNDS(C.status, e, C.S, kSiteSorted)) break;
          const bool two = e + 1 < e1 && VX_IN_BOUNDS(C.status, e + 1, C.S, kSiteSorted);
          const int4 ca = C.scell[e], fa = C.sinf[e];
          int4 cb = ca, fb = fa;
          if (two) { cb = C.scell[e + 1]; fb = C.sinf[e + 1]; }
          take(e, ca, fa);
          if (two) take(e + 1, cb, fb);
        }
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
  if (C.vcnt) C.vcnt[v] = n;
  if (overflow) atomicOr(C.status, kStatusCapacity);
}

// Candidates of searched voxel s, found by one warp: lane l < 27 scans the
// hash bucket of neighbour cell l (dx, dy, dz = l mod 3, l / 3 mod 3, l / 9,
// each minus 1), so a search costs one bucket's chain of loads instead of
// 27 in a row.  The lanes' finds are gathered in the warp's shared buffer
// (kCandCap ints), sorted ascending by canonical index and written out.  A
// lane holds at most kLaneCap finds (a cell of non-overlapping voxels holds
// at most 8); if a cell yields more, lane 0 searches the voxel again alone
// (query_one), so the lists and the overflow report are those of the
// 48-candidate limit either way.
constexpr int kLaneCap = 16;

__device__ __forceinline__ void query_warp(const CollideArgs& C, int s, int lane, int* buf) {
  const int v = C.surf[s];
  const int b = C.body ? C.body[v] : 0;
  if (!C.flag[b]) return;  // the same s for the whole warp
  const int64_t x0 = C.xq[s], y0 = C.xq[(int64_t)C.S + s], z0 = C.xq[2 * (int64_t)C.S + s];
  const int64_t cs = 2 * C.Q;
  const int4 c0 = C.cell[s];
  const uint32_t lp = C.lat[v];
  const int vi = (int)(lp & 2047u), vj = (int)((lp >> 11) & 2047u), vk = (int)(lp >> 22);
  const int64_t r2max = cs * cs;  // (2 Q)^2
  int mine[kLaneCap];
  int n = 0;
  bool overflow = false;
  if (lane < 27) {
    const int ncx = c0.x + lane % 3 - 1, ncy = c0.y + (lane / 3) % 3 - 1, ncz = c0.z + lane / 9 - 1;
    const uint32_t h = cell_hash(ncx, ncy, ncz, C.H - 1);
    const uint32_t e0 = C.hstart[h], e1 = C.hstart[h + 1];
    auto take = [&](uint32_t e, int4 c1, int4 f) {
      if (c1.w == s) return;
      if (c1.x != ncx || c1.y != ncy || c1.z != ncz) return;  // another cell in the same bucket
      const int u = f.x;
      if (C.body && f.z != b) {
        if (!C.qorg) return;  // bodies are separate worlds
      } else {
        const uint32_t lq = (uint32_t)f.y;
        const int man = abs((int)(lq & 2047u) - vi) + abs((int)((lq >> 11) & 2047u) - vj) + abs((int)(lq >> 22) - vk);
        if (man <= 3) return;
      }
      const int64_t x1 = C.sxq[e], y1 = C.sxq[(int64_t)C.S + e], z1 = C.sxq[2 * (int64_t)C.S + e];
      const int64_t ddx = x1 - x0, ddy = y1 - y0, ddz = z1 - z0;
      if (ddx * ddx + ddy * ddy + ddz * ddz >= r2max) return;
      if (n < kLaneCap) mine[n++] = u; else overflow = true;
    };
    for (uint32_t e = e0; e < e1; e += 2) {  // two entries requested at once
      if (!VX_IN_BOUNDS(C.status, e, C.S, kSiteSorted)) break;
      const bool two = e + 1 < e1 && VX_IN_BOUNDS(C.status, e + 1, C.S, kSiteSorted);
      const int4 ca = C.scell[e], fa = C.sinf[e];
      int4 cb = ca, fb = fa;
      if (two) { cb = C.scell[e + 1]; fb = C.sinf[e + 1]; }
      take(e, ca, fa);
      if (two) take(e + 1, cb, fb);
    }
  }
  if (__any_sync(0xffffffffu, overflow)) {  // a crowded cell: the one-thread search
    if (lane == 0) query_one(C, s);
    __syncwarp();
    return;
  }
  // offsets of the lanes' finds in the buffer (prefix sum over the warp)
  int inc = n;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  const int total = __shfl_sync(0xffffffffu, inc, 31);
  const int off = inc - n;
  for (int i = 0; i < n; ++i)
    if (off + i < kCandCap) buf[off + i] = mine[i];
  if (total > kCandCap) overflow = true;
  __syncwarp();
  const int m = total < kCandCap ? total : kCandCap;
  if (lane == 0)
    for (int i = 1; i < m; ++i) {  // insertion sort ascending (lists are short)
      const int x = buf[i];
      int k = i - 1;
      while (k >= 0 && buf[k] > x) { buf[k + 1] = buf[k]; --k; }
      buf[k + 1] = x;
    }
  __syncwarp();
  int32_t* out = C.cand + (int64_t)s * kCandCap;
  for (int i = lane; i < m; i += 32) out[i] = buf[i];
  if (lane == 0) {
    C.ccount[s] = m;
    if (C.vcnt) C.vcnt[v] = m;
  }
  if (__any_sync(0xffffffffu, overflow) && lane == 0) atomicOr(C.status, kStatusCapacity);
  __syncwarp();  // the buffer is reused for the warp's next voxel
}

constexpr int kWarpWs = kCandCap;  // ints of query workspace per warp

// The rebuild phases, run by every CTA of a cooperative grid (any number of
// CTAs up to kRebuildMaxGrid, blockDim a multiple of 32 up to 1024); G is
// the count the grid barriers wait for; ws: shared-memory workspace of
// kWarpWs ints per warp.  Returns false if a barrier wait gave up.
__device__ __forceinline__ bool rebuild_phases(const CollideArgs& C, unsigned G, int* ws) {
  __shared__ uint32_t warp_tot[32];
  __shared__ uint32_t offset;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
  // zero the bucket counters
  for (int i = tid; i < C.H; i += nthr) { C.hcount[i] = 0u; C.hcursor[i] = 0u; }
  if (!grid_barrier(C.bar, G, C.spins, C.status)) return false;
  for (int s = tid; s < C.S; s += nthr) quantise_one(C, s);
  if (!grid_barrier(C.bar, G, C.spins, C.status)) return false;
  // scan: CTA c owns buckets [c chunk, (c + 1) chunk)
  const int chunk = (C.H + (int)gridDim.x - 1) / (int)gridDim.x;
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
  if (!grid_barrier(C.bar, G, C.spins, C.status)) return false;
  {
    // offset of this CTA's chunk: sum of the chunk totals before it (fixed order)
    uint32_t part = 0u;
    for (int c = threadIdx.x; c < (int)blockIdx.x; c += blockDim.x) part += C.bsum[c];
    uint32_t tot;
    block_exclusive_scan(part, warp_tot, &tot);
    if (threadIdx.x == 0) offset = tot;
    __syncthreads();
    for (int i = b0 + threadIdx.x; i < b1; i += blockDim.x) C.hstart[i] += offset;
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) C.hstart[C.H] = offset + carry;
  }
  if (!grid_barrier(C.bar, G, C.spins, C.status)) return false;
  for (int s = tid; s < C.S; s += nthr) {
    const uint32_t h = C.bucket[s];
    if (!VX_IN_BOUNDS(C.status, h, C.H, kSiteBucket)) continue;
    const uint32_t at = C.hstart[h] + atomicAdd(&C.hcursor[h], 1u);
    if (!VX_IN_BOUNDS(C.status, at, C.S, kSiteSorted)) continue;
    C.sorted[at] = s;
    // the query reads each bucket's entries as one contiguous run
    const int4 c = C.cell[s];
    C.scell[at] = make_int4(c.x, c.y, c.z, s);
    for (int a = 0; a < 3; ++a) C.sxq[(int64_t)a * C.S + at] = C.xq[(int64_t)a * C.S + s];
    const int u = C.surf[s];
    C.sinf[at] = make_int4(u, (int)C.lat[u], C.body ? C.body[u] : 0, 0);
  }
  if (!grid_barrier(C.bar, G, C.spins, C.status)) return false;
  {
    // one warp per searched voxel while that leaves at most 8 voxels to a
    // warp (8 one-cell chains of dependent loads, against one 27-cell chain
    // per thread); beyond, one thread per voxel (the search is bound by the
    // latency of its chains, so the most independent chains win).  Both
    // give the same sorted lists.
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nw = (int)(gridDim.x * (blockDim.x >> 5));
    if (C.S <= 8 * nw) {
      for (int q = (int)blockIdx.x * (int)(blockDim.x >> 5) + w; q < C.S; q += nw) query_warp(C, q, lane, ws + w * kWarpWs);
    } else {
      for (int q = tid; q < C.S; q += nthr) query_one(C, q);
    }
  }
  if (!grid_barrier(C.bar, G, C.spins, C.status)) return false;
  if (blockIdx.x == 0) {
    for (int b = threadIdx.x; b < C.n_bodies; b += blockDim.x) C.flag[b] = 0;
    __syncthreads();
    if (threadIdx.x == 0) { *C.any = 0; *C.n_rebuilds += 1; }
  }
  return true;
}

}  // namespace vx

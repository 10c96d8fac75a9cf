// Collision candidates without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need
// collision candidates: code running inside a memory pool or arena that owns
// every byte of the device heap, a plug-in given only pre-sized buffers by its
// host application, or an allocator-free real-time loop where cudaMalloc's
// implicit synchronisation is not acceptable.  vx_collision_candidates_static
// serves them: the caller passes the surface voxels and the output lists, and
// the hash grid and sort buffers come from one fixed array in this file.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds it (kScratchBytes, about 8.3 MiB) until the process exits.  Host
// code cannot use the array's name as a device address, so the first call on
// each device, with that device current, looks up the address with
// cudaGetSymbolAddress and keeps it for later calls.  Make that first call
// before any stream capture.  All calls share the array: calls whose GPU work
// overlaps (different streams, or different host threads on one device) race
// on it and must be serialised by the caller.  Each call clears what the
// pipeline needs cleared, so the contents left by the previous call never
// matter.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "vx.h"
#include "vx_host.h"
#include "vx_kernels.h"

namespace vx {
namespace {

constexpr int64_t kMaxSurface = VX_STATIC_MAX_SURFACE;
constexpr int64_t kMaxBodies = VX_STATIC_MAX_BODIES;
constexpr int64_t kMaxBuckets = 2 * kMaxSurface;  // power of two, >= 2 S

constexpr size_t align256(size_t n) { return (n + 255) / 256 * 256; }
constexpr size_t kOffXq = 0;
constexpr size_t kOffCell = kOffXq + align256(3 * kMaxSurface * sizeof(int64_t));
constexpr size_t kOffBucket = kOffCell + align256(kMaxSurface * sizeof(int4));
constexpr size_t kOffCount = kOffBucket + align256(kMaxSurface * sizeof(uint32_t));
constexpr size_t kOffCursor = kOffCount + align256(kMaxBuckets * sizeof(uint32_t));
constexpr size_t kOffStart = kOffCursor + align256(kMaxBuckets * sizeof(uint32_t));
constexpr size_t kOffBsum = kOffStart + align256((kMaxBuckets + 1) * sizeof(uint32_t));
constexpr size_t kOffSorted = kOffBsum + align256(kRebuildMaxGrid * sizeof(uint32_t));
constexpr size_t kOffScell = kOffSorted + align256(kMaxSurface * sizeof(int32_t));
constexpr size_t kOffSxq = kOffScell + align256(kMaxSurface * sizeof(int4));
constexpr size_t kOffSinf = kOffSxq + align256(3 * kMaxSurface * sizeof(int64_t));
constexpr size_t kOffIota = kOffSinf + align256(kMaxSurface * sizeof(int4));
constexpr size_t kOffAcc = kOffIota + align256(kMaxSurface * sizeof(int32_t));
constexpr size_t kOffFlag = kOffAcc + align256(kMaxBodies * sizeof(float));
constexpr size_t kOffMisc = kOffFlag + align256(kMaxBodies * sizeof(int));  // any, status[8], n_rebuilds, barrier
constexpr size_t kScratchBytes = kOffMisc + 256;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

int fail(int code, const std::string& m) { return set_error(code, m); }

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device (looked up once per device).
int scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(VX_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(VX_ERR_CUDA, "device index out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p)
      return fail(VX_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_addr[dev];
  return VX_OK;
}

// Identity surface list; body ids outside [0, n_bodies) set the argument
// status bit and record the first offending input index.
__global__ void prepare_kernel(int32_t* a, int n, const int32_t* body, int n_bodies, int* status) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  a[i] = i;
  if (body) {
    const int b = body[i];
    if (b < 0 || b >= n_bodies) {
      atomicOr(status, kStatusArg);
      atomicMin(status + 1, i);
    }
  }
}

}  // namespace
}  // namespace vx

using namespace vx;

extern "C" VX_API int vx_collision_candidates_static(const uint32_t* lat, const float* offset_planes,
                                                     const int32_t* body, int32_t n_surface, int32_t n_bodies,
                                                     float voxel_size, int32_t* cand_count, int32_t* cand,
                                                     void* stream) {
  if (n_surface < 0 || n_surface > kMaxSurface)
    return fail(VX_ERR_ARG, "n_surface must be in [0, " + std::to_string(kMaxSurface) + "], got " +
                                std::to_string(n_surface));
  if (n_bodies < 1 || n_bodies > kMaxBodies)
    return fail(VX_ERR_ARG, "n_bodies must be in [1, " + std::to_string(kMaxBodies) + "], got " +
                                std::to_string(n_bodies));
  if (!(voxel_size > 0.f)) return fail(VX_ERR_ARG, "voxel_size must be positive");
  if (n_surface > 0 && (!lat || !offset_planes || !cand_count || !cand))
    return fail(VX_ERR_ARG, "lat, offset_planes, cand_count and cand are required");
  if (n_bodies > 1 && n_surface > 0 && !body) return fail(VX_ERR_ARG, "body is required when n_bodies > 1");
  if (n_surface == 0) return VX_OK;
  unsigned char* base = nullptr;
  int rc = scratch_address(&base);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  int H = 1024;
  while ((int64_t)H < 2 * (int64_t)n_surface) H <<= 1;
  CollideArgs C;
  C.S = n_surface;
  C.n_bodies = n_bodies;
  C.H = H;
  quant_params(voxel_size, &C.K, &C.Q);
  C.ostride_v = 1;                     // offset planes: x[S], y[S], z[S]
  C.ostride_a = n_surface;
  C.threshold = 0.f;
  C.st = offset_planes;
  C.surf = reinterpret_cast<int32_t*>(base + kOffIota);  // identity: surface index = voxel index
  C.lat = lat;
  C.body = n_bodies > 1 ? body : nullptr;
  C.dt_body = nullptr;
  C.xq = reinterpret_cast<int64_t*>(base + kOffXq);
  C.cell = reinterpret_cast<int4*>(base + kOffCell);
  C.bucket = reinterpret_cast<uint32_t*>(base + kOffBucket);
  C.hcount = reinterpret_cast<uint32_t*>(base + kOffCount);
  C.hcursor = reinterpret_cast<uint32_t*>(base + kOffCursor);
  C.hstart = reinterpret_cast<uint32_t*>(base + kOffStart);
  C.bsum = reinterpret_cast<uint32_t*>(base + kOffBsum);
  C.sorted = reinterpret_cast<int32_t*>(base + kOffSorted);
  C.scell = reinterpret_cast<int4*>(base + kOffScell);
  C.sxq = reinterpret_cast<int64_t*>(base + kOffSxq);
  C.sinf = reinterpret_cast<int4*>(base + kOffSinf);
  C.ccount = cand_count;
  C.vcnt = nullptr;
  C.cand = cand;
  C.acc = reinterpret_cast<float*>(base + kOffAcc);
  C.vmax_bits = nullptr;
  C.flag = reinterpret_cast<int*>(base + kOffFlag);
  C.any = reinterpret_cast<int*>(base + kOffMisc);
  C.status = reinterpret_cast<int*>(base + kOffMisc + 16);
  C.n_rebuilds = reinterpret_cast<long long*>(base + kOffMisc + 64);
  C.bar = reinterpret_cast<unsigned*>(base + kOffMisc + 128);
  C.qorg = nullptr;
  C.spins = 1ll << 24;
  // status words: bits, then the first out-of-range body index (starts at
  // 0x7F7F7F7F, above any input index)
  cudaError_t e = cudaMemsetAsync(C.status, 0, 32, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(C.status + 1, 0x7F, 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(C.bar, 0, 2 * sizeof(unsigned), st);
  if (e != cudaSuccess) return fail(VX_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  prepare_kernel<<<(n_surface + 255) / 256, 256, 0, st>>>(const_cast<int32_t*>(C.surf), n_surface, C.body,
                                                          n_bodies, C.status);
  int status[4] = {0, 0, 0, 0};
  // the body ids are checked before the rebuild indexes per-body scratch with them
  if (C.body && ((e = cudaGetLastError()) != cudaSuccess ||
                 (e = cudaMemcpyAsync(status, C.status, 16, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
                 (e = cudaStreamSynchronize(st)) != cudaSuccess))
    return fail(VX_ERR_CUDA, std::string("collision candidates: ") + cudaGetErrorString(e));
  if (status[0] & kStatusArg)
    return fail(VX_ERR_ARG, "body id out of [0, n_bodies) at surface voxel " + std::to_string(status[1]));
  launch_flag_all(C, st);
  launch_rebuild(C, st);
  if ((e = cudaGetLastError()) != cudaSuccess ||
      (e = cudaMemcpyAsync(status, C.status, 16, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return fail(VX_ERR_CUDA, std::string("collision candidates: ") + cudaGetErrorString(e));
  if (status[0] & kStatusTimeout) return fail(VX_ERR_TIMEOUT, "a grid barrier of the candidate search gave up waiting");
  if (status[0] & kStatusBounds) return fail(VX_ERR_BOUNDS, "an index failed its bounds check (debug build)");
  if (status[0] & kStatusCapacity)
    return fail(VX_ERR_CAPACITY, "more than " + std::to_string(kCandCap) + " candidates for a surface voxel");
  return VX_OK;
}

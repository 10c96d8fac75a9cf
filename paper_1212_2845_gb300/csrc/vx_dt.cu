// Stable timestep of every body (Sec 2.1.4) as a device max-reduction in
// FP32, the precision the step itself runs in.
//
// The largest w^2 = k / m of a body is taken over every voxel's own contact
// spring, E_v l / m_v, and every bond to a +a neighbour, E_c l / min(m_v, m_u)
// with E_c = 2 E_v E_u / (E_v + E_u).  Each CTA takes one chunk of one
// body's internal range; the threads' maxima meet in a warp shuffle, then
// across the warps in shared memory, then one atomicMax per CTA on the bits
// of the non-negative float (their integer order is the numeric order).  A
// candidate that is NaN (0 / 0 for two zero moduli) is skipped, since a
// comparison with it is false; an infinite one wins (dt = 0 follows).
#include "vx_dev.cuh"
#include "vx_kernels.h"

namespace vx {
namespace {

__device__ __forceinline__ float modulus(const DtArgs& D, int v, int m) {
  return D.logE ? expf(D.logE[v]) : D.mats[m].E;
}

__global__ void __launch_bounds__(kDtThreads) stable_w2(DtArgs D) {
  const int4 c = D.chunks[blockIdx.x];
  float w = 0.f;
  for (int v = c.x + (int)threadIdx.x; v < c.y; v += blockDim.x) {
    const int iv = D.mat[v];
    const float Ev = modulus(D, v, iv), mv = D.mats[iv].m;
    float x = __fdiv_rn(__fmul_rn(Ev, D.l), mv);
    if (x > w) w = x;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int u = D.nbr[(int64_t)(2 * a + 1) * D.N + v];
      if (u < 0) continue;
      const int iu = D.mat[u];
      const float Eu = modulus(D, u, iu), mu = D.mats[iu].m;
      const float Ec = __fdiv_rn(__fmul_rn(__fmul_rn(2.f, Ev), Eu), __fadd_rn(Ev, Eu));
      x = __fdiv_rn(__fmul_rn(Ec, D.l), fminf(mv, mu));
      if (x > w) w = x;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float y = __shfl_xor_sync(0xffffffffu, w, o);
    if (y > w) w = y;
  }
  __shared__ float red[kDtThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = w;
  __syncthreads();
  if (warp == 0) {
    w = lane < kDtThreads / 32 ? red[lane] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float y = __shfl_xor_sync(0xffffffffu, w, o);
      if (y > w) w = y;
    }
    if (lane == 0) atomicMax(&D.w2[c.z], __float_as_uint(w));
  }
}

}  // namespace

void launch_stable_w2(const DtArgs& D, cudaStream_t s) {
  if (D.n_chunks > 0) stable_w2<<<D.n_chunks, kDtThreads, 0, s>>>(D);
}

}  // namespace vx

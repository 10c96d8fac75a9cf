// Shared-memory-resident multi-step form (same arithmetic, same bits as the
// per-step kernels).
//
// A group of whole bodies lives in the shared memory of one CTA cluster for
// all n steps of a launch: each CTA of the cluster holds a contiguous slice
// of the group's voxels (state, bond results, material properties, the
// neighbour table), loaded once at the start and written back once at the
// end.  A step is two phases separated by cluster barriers, in one of two
// work splits:
//
//   BOND (latency: a small lattice spread over a cluster)
//     bonds   one thread per bond (voxel u, lattice axis a, u on the
//             negative side) evaluates the co-rotational beam with the
//             partner's state read from whichever CTA of the cluster holds it
//             (distributed shared memory) and stores F1, M1, M2 in u's slot;
//     voxels  one thread per voxel sums its +x, +y, +z slots and the -x, -y,
//             -z slots of its neighbours in the order of the per-step kernels
//             and runs the voxel update;
//   VOXEL (throughput: many groups)
//     bonds   one thread per voxel evaluates its own +x, +y, +z bonds with its
//             rotation matrix computed once, keeps the sums of F1 and M1 in
//             its own slot and stores F1, M2 for the partners;
//     voxels  the same voxel adds its neighbours' -x, -y, -z results and runs
//             the voxel update.
//
// Either way every bond is evaluated once (no halo copies), the state is
// updated in place, and the voxel's thermal strain for the next step is
// written at the end of the voxel phase.  No bond result, state or property
// touches global memory between the two loads, and no grid-wide barrier or
// launch separates the steps.  Clusters take their groups one after the
// other (longest first onto the least loaded cluster, planned on the host);
// there are no voxel-voxel collisions in this form (bodies are independent
// worlds; the floor is fine).
#include <cooperative_groups.h>

#include "vx_dev.cuh"
#include "vx_kernels.h"

namespace vx {
namespace cg = cooperative_groups;
namespace {

constexpr int kLocBits = 11;                 // neighbour entry: rank << 11 | local slot
constexpr uint16_t kNoNb = 0xFFFF;

// One CTA's slice of a group in shared memory (capacity V voxels).  Bond
// slots are [3][V] per array, axis-major: sa (F1.x, F1.y, F1.z, M2.x),
// sb (M2.y, M2.z, M1.x, M1.y), sc M1.z, so a neighbour's -a gather (F1 and
// M2) reads one float4 and one float2.  The VOXEL split stores no M1 per
// bond; there the voxel's own sums F and M of its +x, +y, +z bonds take the
// freed places: F.x, F.y in the last two floats of sb[2V + u], F.z in
// sc[u], M.x in sc[V + u], M.y in sc[2V + u], M.z in sb[V + u].z.
struct ResSmem {
  float4 *A, *B, *C;   // state planes (as in global memory)
  float* D;
  float4 *sa, *sb;     // bond slots
  float* sc;
  float4* pr;          // E, G, thermal strain of the current step, material (bits)
  uint16_t* nb;        // [6][V]: -x, +x, -y, +y, -z, +z neighbour or kNoNb
  float *z0, *dt, *ph; // anchor height of the centre, body timestep, actuation phase
  float* fx;           // 3 x V external force (null when unused)
  uint8_t* fl;         // flags
  DevMat* mats;
  float* lut;

  static __host__ __device__ size_t bytes(int V, bool fext, int n_mats, bool lut) {
    return (size_t)V * (3 * 16 + 4 + 2 * 3 * 16 + 3 * 4 + 16 + 6 * 2 + 3 * 4 + (fext ? 12 : 0) + 1) + 16 +
           (size_t)n_mats * sizeof(DevMat) + (lut ? (size_t)8 * n_mats * n_mats * 4 : 0);
  }
  __device__ __forceinline__ void carve(float* base, int V, bool fext, int n_mats, bool has_lut) {
    A = reinterpret_cast<float4*>(base);
    B = A + V;
    C = B + V;
    sa = C + V;
    sb = sa + 3 * V;
    pr = sb + 3 * V;
    float* p = reinterpret_cast<float*>(pr + V);
    D = p; p += V;
    sc = p; p += 3 * V;
    z0 = p; p += V;
    dt = p; p += V;
    ph = p; p += V;
    fx = fext ? p : nullptr; p += fext ? 3 * V : 0;
    mats = reinterpret_cast<DevMat*>(p);                 // 4-byte fields
    lut = reinterpret_cast<float*>(mats + n_mats);
    // the LUT is read as float4: round its start up to 16 bytes
    lut = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(lut) + 15) & ~uintptr_t(15));
    nb = reinterpret_cast<uint16_t*>(lut + (has_lut ? 8 * n_mats * n_mats : 0));
    fl = reinterpret_cast<uint8_t*>(nb + 6 * V);
  }
  __device__ __forceinline__ VoxS vox(int k) const { return unpack_vox(A[k], B[k], C[k], D[k]); }
  __device__ __forceinline__ void put(int k, const VoxS& s) const {
    A[k] = make_float4(s.o.x, s.o.y, s.o.z, s.q.w);
    B[k] = make_float4(s.q.x, s.q.y, s.q.z, s.v.x);
    C[k] = make_float4(s.v.y, s.v.z, s.w.x, s.w.y);
    D[k] = s.w.z;
  }
};


// State and properties of slot k2 of cluster rank r2 through distributed
// shared memory; with LOCAL, plain shared-memory loads when it is this CTA
// (a branch that pays where most partners are local: large slices).
template <bool LOCAL>
__device__ __forceinline__ void partner(const cg::cluster_group& cl, const ResSmem& S, int rank, int r2, int k2,
                                        VoxS& s2, float4& p2) {
  if (LOCAL && r2 == rank) {
    s2 = S.vox(k2);
    p2 = S.pr[k2];
    return;
  }
  const float4* A2 = cl.map_shared_rank(S.A, r2);
  const float4* B2 = cl.map_shared_rank(S.B, r2);
  const float4* C2 = cl.map_shared_rank(S.C, r2);
  const float* D2 = cl.map_shared_rank(S.D, r2);
  s2 = unpack_vox(A2[k2], B2[k2], C2[k2], D2[k2]);
  p2 = cl.map_shared_rank(S.pr, r2)[k2];
}

// F1 and M2 of the -a bond of a voxel, stored by its neighbour (slot k2 of rank r2).
template <bool LOCAL>
__device__ __forceinline__ void minus_result(const cg::cluster_group& cl, const ResSmem& S, int rank, int r2, int k2,
                                             int a, int V, float4& f, float2& h) {
  if (LOCAL && r2 == rank) {
    f = S.sa[a * V + k2];
    h = *reinterpret_cast<const float2*>(S.sb + a * V + k2);
    return;
  }
  f = cl.map_shared_rank(S.sa, r2)[a * V + k2];
  h = *reinterpret_cast<const float2*>(cl.map_shared_rank(S.sb, r2) + a * V + k2);
}

__device__ __forceinline__ BondK res_consts(const StepArgs& A, const ResSmem& S, float4 p1, float4 p2) {
  const int m1 = __float_as_int(p1.w), m2 = __float_as_int(p2.w);
  if (A.lut) return lut_consts(S.lut, A.n_mats, m1, m2);
  return bond_consts(A.l, p1.x, p2.x, p1.y, p2.y, fminf(S.mats[m1].m, S.mats[m2].m), fminf(S.mats[m1].I, S.mats[m2].I),
                     A.zb);
}

template <bool FX, bool PER_VOXEL>
__global__ void __launch_bounds__(kResThreads, 1) res_pipe(StepArgs A0, ResArgs R) {
  extern __shared__ __align__(16) float smem[];
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int C = (int)cl.num_blocks();
  const int cid = (int)blockIdx.x / C;
  const int V = R.cap, T = (int)blockDim.x, tid = (int)threadIdx.x;
  ResSmem S;
  S.carve(smem, V, FX, A0.n_mats, A0.lut != nullptr);
  for (int j = tid; j < A0.n_mats * (int)(sizeof(DevMat) / 4); j += T)
    reinterpret_cast<float*>(S.mats)[j] = reinterpret_cast<const float*>(A0.mats)[j];
  if (A0.lut)
    for (int j = tid; j < 8 * A0.n_mats * A0.n_mats; j += T) S.lut[j] = A0.lut[j];
  const int64_t step0 = R.ctr ? R.ctr[0] : R.step0;
  const int cur0 = R.ctr ? (int)R.ctr[1] : R.cur0;
  const float* st_in = cur0 ? R.buf1 : R.buf0;
  float* st_out = ((cur0 + R.n_steps) & 1) ? R.buf1 : R.buf0;
  const int64_t P = A0.pitch;
  const bool damp = A0.zb != 0.f;
  __syncthreads();
  for (int gi = R.cl_start[cid]; gi < R.cl_start[cid + 1]; ++gi) {
    const int g = R.cl_groups[gi];
    const int g0 = R.grp_start[g], n = R.grp_start[g + 1] - g0;
    const int slice = (n + C - 1) / C;
    const int u0 = g0 + rank * slice;
    const int ns = max(0, min(slice, g0 + n - u0));
    // ---- load the slice: state at step0, properties at step0, neighbours
    {
      StepArgs A = A0;
      A.act_w = act_angle(step0, R.act_P, R.act_c);
      const StPtr G(const_cast<float*>(st_in), P);
      for (int u = tid; u < ns; u += T) {
        const int v = u0 + u;
        S.A[u] = G.A[v];
        S.B[u] = G.B[v];
        S.C[u] = G.C[v];
        S.D[u] = G.D[v];
        const int m = A0.mat[v];
        const DevMat& d = S.mats[m];
        const float ph = A0.phase ? A0.phase[v] : 0.f;
        S.ph[u] = ph;
        const float E = A0.logE ? expf(A0.logE[v]) : d.E;
        S.pr[u] = make_float4(E, __fmul_rn(E, d.g_ratio), strain_of(A, d, ph), __int_as_float(m));
        for (int sl = 0; sl < 6; ++sl) {
          const int j = A0.nbr[(int64_t)sl * A0.N + v];
          uint16_t e = kNoNb;
          if (j >= 0) {
            const int k = j - g0, r = k / slice;
            e = (uint16_t)((r << kLocBits) | (k - r * slice));
          }
          S.nb[sl * V + u] = e;
        }
        const uint32_t lp = A0.lat[v];
        const int b = A0.body ? A0.body[v] : 0;
        S.z0[u] = fma_(add_((float)(int)(lp >> 22), 0.5f), A0.l, A0.origin[3 * b + 2]);
        S.dt[u] = A0.dt_body[b];
        S.fl[u] = A0.flags[v];
        if (FX) {
          S.fx[u] = A0.fext[v];
          S.fx[V + u] = A0.fext[P + v];
          S.fx[2 * V + u] = A0.fext[2 * P + v];
        }
      }
    }
    cl.sync();
    for (int k = 0; k < R.n_steps; ++k) {
      StepArgs A = A0;
      A.step = step0 + k;
      if (!PER_VOXEL) {
        // ---- bonds: thread per (axis, voxel) with the voxel on the negative side
        for (int bi = tid; bi < 3 * ns; bi += T) {
          const int a = (bi >= ns) + (bi >= 2 * ns);
          const int u = bi - a * ns;
          const uint16_t e = S.nb[(2 * a + 1) * V + u];
          if (e == kNoNb || !VX_IN_BOUNDS(A.status, e >> kLocBits, C, kSiteCluster) ||
              !VX_IN_BOUNDS(A.status, e & ((1 << kLocBits) - 1), slice, kSiteCluster))
            continue;
          VoxS s2;
          float4 p2;
          partner<false>(cl, S, rank, e >> kLocBits, e & ((1 << kLocBits) - 1), s2, p2);
          const VoxS s1 = S.vox(u);
          const float4 p1 = S.pr[u];
          const BondOut o = bond_eval_r(s1, qmat(s1.q), s2, A.l, res_consts(A, S, p1, p2),
                                        mul_(0.5f, add_(p1.z, p2.z)), damp, a);
          S.sa[a * V + u] = make_float4(o.F1.x, o.F1.y, o.F1.z, o.M2.x);
          S.sb[a * V + u] = make_float4(o.M2.y, o.M2.z, o.M1.x, o.M1.y);
          S.sc[a * V + u] = o.M1.z;
        }
      } else {
        // ---- bonds: thread per voxel, its own +x, +y, +z bonds
        for (int u = tid; u < ns; u += T) {
          const VoxS s1 = S.vox(u);
          const float4 p1 = S.pr[u];
          const M3f R1 = qmat(s1.q);
          V3f F = v3(0.f, 0.f, 0.f), M = v3(0.f, 0.f, 0.f);
#define VX_RES_BOND(AX)                                                                                     \
          {                                                                                                 \
            const uint16_t e = S.nb[(2 * AX + 1) * V + u];                                                  \
            if (e != kNoNb && VX_IN_BOUNDS(A.status, e >> kLocBits, C, kSiteCluster) &&                      \
                VX_IN_BOUNDS(A.status, e & ((1 << kLocBits) - 1), slice, kSiteCluster)) {                   \
              VoxS s2;                                                                                      \
              float4 p2;                                                                                    \
              partner<true>(cl, S, rank, e >> kLocBits, e & ((1 << kLocBits) - 1), s2, p2);                 \
              const BondOut o = bond_eval<AX>(s1, R1, s2, A.l, res_consts(A, S, p1, p2),                    \
                                              mul_(0.5f, add_(p1.z, p2.z)), damp);                           \
              F = add(F, o.F1);                                                                             \
              M = add(M, o.M1);                                                                             \
              S.sa[AX * V + u] = make_float4(o.F1.x, o.F1.y, o.F1.z, o.M2.x);                               \
              *reinterpret_cast<float2*>(S.sb + AX * V + u) = make_float2(o.M2.y, o.M2.z);                  \
            }                                                                                               \
          }
          VX_RES_BOND(0)
          VX_RES_BOND(1)
          VX_RES_BOND(2)
#undef VX_RES_BOND
          // own sums in the unused halves of the z-axis plane of sb and in sc
          reinterpret_cast<float2*>(S.sb + 2 * V + u)[1] = make_float2(F.x, F.y);
          S.sc[u] = F.z;
          S.sc[V + u] = M.x;
          S.sc[2 * V + u] = M.y;
          reinterpret_cast<float2*>(S.sb + V + u)[1] = make_float2(M.z, 0.f);
        }
      }
      cl.sync();
      // ---- voxels: the per-step kernels' summation order (+x, +y, +z own
      // bonds, then the -x, -y, -z bonds of the neighbours), then the update
      const float w_next = act_angle(step0 + k + 1, R.act_P, R.act_c);
      for (int u = tid; u < ns; u += T) {
        V3f F, M;
        if (!PER_VOXEL) {
          F = v3(0.f, 0.f, 0.f);
          M = v3(0.f, 0.f, 0.f);
#pragma unroll
          for (int a = 0; a < 3; ++a)
            if (S.nb[(2 * a + 1) * V + u] != kNoNb) {
              const float4 f = S.sa[a * V + u], h = S.sb[a * V + u];
              F = add(F, v3(f.x, f.y, f.z));
              M = add(M, v3(h.z, h.w, S.sc[a * V + u]));
            }
        } else {
          const float2 fxy = reinterpret_cast<const float2*>(S.sb + 2 * V + u)[1];
          const float2 mz = reinterpret_cast<const float2*>(S.sb + V + u)[1];
          F = v3(fxy.x, fxy.y, S.sc[u]);
          M = v3(S.sc[V + u], S.sc[2 * V + u], mz.x);
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const uint16_t e = S.nb[2 * a * V + u];
          if (e != kNoNb && VX_IN_BOUNDS(A.status, e >> kLocBits, C, kSiteCluster) &&
              VX_IN_BOUNDS(A.status, e & ((1 << kLocBits) - 1), slice, kSiteCluster)) {
            float4 f;
            float2 h;
            minus_result<PER_VOXEL>(cl, S, rank, e >> kLocBits, e & ((1 << kLocBits) - 1), a, V, f, h);
            F = sub(F, v3(f.x, f.y, f.z));  // F - F1 is F + (-F1) exactly
            M = add(M, v3(f.w, h.x, h.y));
          }
        }
        const float4 p = S.pr[u];
        VoxMeta mt;
        mt.lat = 0u;
        mt.m = __float_as_int(p.w);
        mt.b = 0;
        mt.fl = S.fl[u];
        mt.dt = S.dt[u];
        mt.z0 = S.z0[u];
        mt.fext = FX ? v3(S.fx[u], S.fx[V + u], S.fx[2 * V + u]) : v3(0.f, 0.f, 0.f);
        mt.nc = 0;
        VoxS s = S.vox(u);
        uint8_t fl;
        voxel_update(A, u0 + u, mt, s, fl, F, M, p.z, p.x, S.mats);
        S.put(u, s);
        S.fl[u] = fl;
        // thermal strain of the next step
        A.act_w = w_next;
        S.pr[u].z = strain_of(A, S.mats[mt.m], S.ph[u]);
      }
      cl.sync();
    }
    // ---- write the slice back (state after n steps, flags)
    {
      const StPtr G(st_out, P);
      for (int u = tid; u < ns; u += T) {
        const int v = u0 + u;
        G.A[v] = S.A[u];
        G.B[v] = S.B[u];
        G.C[v] = S.C[u];
        G.D[v] = S.D[u];
        A0.flags[v] = S.fl[u];
      }
    }
  }
}

cudaLaunchConfig_t res_config(int grid, int C, int threads, size_t smem, cudaStream_t s, cudaLaunchAttribute* at) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cfg;
}

template <bool FX, bool PV> int prepare_res_t(int C, int threads, size_t smem, int* max_clusters) {
  auto* k = res_pipe<FX, PV>;
  cudaError_t e = allow_smem(k, smem);
  if (e == cudaSuccess && C > 8) e = cudaFuncSetAttribute((const void*)k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) { cudaGetLastError(); return -1; }
  cudaLaunchAttribute at[1];
  cudaLaunchConfig_t cfg = res_config(C, C, threads, smem, 0, at);
  int n = 0;
  e = cudaOccupancyMaxActiveClusters(&n, (const void*)k, &cfg);
  if (e != cudaSuccess) { cudaGetLastError(); return -1; }
  *max_clusters = n;
  return n > 0 ? 0 : -1;
}

}  // namespace

size_t res_smem_bytes(int cap, bool fext, int n_mats, bool lut) { return ResSmem::bytes(cap, fext, n_mats, lut); }

int prepare_resident(int C, int threads, size_t smem, bool fext, bool per_voxel, int* max_clusters) {
  if (fext) return per_voxel ? prepare_res_t<true, true>(C, threads, smem, max_clusters)
                             : prepare_res_t<true, false>(C, threads, smem, max_clusters);
  return per_voxel ? prepare_res_t<false, true>(C, threads, smem, max_clusters)
                   : prepare_res_t<false, false>(C, threads, smem, max_clusters);
}

cudaError_t launch_resident(const StepArgs& A, const ResArgs& R, int grid, int C, int threads, size_t smem,
                            bool per_voxel, cudaStream_t s) {
  cudaLaunchAttribute at[1];
  cudaLaunchConfig_t cfg = res_config(grid, C, threads, smem, s, at);
  if (A.fext)
    return per_voxel ? cudaLaunchKernelEx(&cfg, res_pipe<true, true>, A, R) : cudaLaunchKernelEx(&cfg, res_pipe<true, false>, A, R);
  return per_voxel ? cudaLaunchKernelEx(&cfg, res_pipe<false, true>, A, R) : cudaLaunchKernelEx(&cfg, res_pipe<false, false>, A, R);
}

}  // namespace vx

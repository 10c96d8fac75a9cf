// One explicit lattice step (Sec 2.1: all bond forces, then every voxel
// updated synchronously), in two forms that share the same device math and
// produce bitwise-identical states:
//
// fused_step  one kernel per step.  A CTA owns one tile (a run of <= TMAX
//             voxels in brick/Morton order) and stages it with its halo in
//             shared memory.  Each thread evaluates its own voxel's +x, +y, +z
//             bonds (keeping F1, M1 in registers and leaving -F1, M2 in the
//             partner's shared slot); bonds from halo voxels are spread over
//             the CTA; after one barrier each voxel adds its -x, -y, -z slots
//             and integrates.  Bond results never leave shared memory.
// bond_pass + voxel_pass  the plain two-kernel form: one thread per bond
//             writes its result to global memory, one thread per voxel
//             gathers them.  Kept as the reference form of the same step.
#include "vx_dev.cuh"
#include "vx_kernels.h"

namespace vx {

// ---------------------------------------------------------------------------
// two-pass form
// ---------------------------------------------------------------------------
template <int a>
__device__ __forceinline__ void bond_pass_axis(const StepArgs& A, int v) {
  int u = A.nbr[(int64_t)(2 * a + 1) * A.N + v];
  if (u < 0) return;
  const int64_t P = A.pitch;
  VoxS s1 = load_vox(A.st_in, P, v), s2 = load_vox(A.st_in, P, u);
  int m1 = A.mat[v], m2 = A.mat[u];
  const DevMat& d1 = A.mats[m1];
  const DevMat& d2 = A.mats[m2];
  float E1 = voxel_E(A, v, m1), E2 = voxel_E(A, u, m2);
  float eps = mul_(0.5f, add_(thermal_strain(A, v, d1.cte), thermal_strain(A, u, d2.cte)));
  M3f R1 = qmat(s1.q);
  BondOut o = bond_eval<a>(s1, R1, s2, A.l, E1, E2, __fmul_rn(E1, d1.g_ratio), __fmul_rn(E2, d2.g_ratio),
                           fminf(d1.m, d2.m), fminf(d1.I, d2.I), eps, A.zb);
  float* bf = A.bf + (int64_t)a * P + v;
  const int64_t C = 3 * P;
  bf[0 * C] = o.F1.x; bf[1 * C] = o.F1.y; bf[2 * C] = o.F1.z;
  bf[3 * C] = o.M1.x; bf[4 * C] = o.M1.y; bf[5 * C] = o.M1.z;
  bf[6 * C] = o.M2.x; bf[7 * C] = o.M2.y; bf[8 * C] = o.M2.z;
}

__global__ void __launch_bounds__(256) bond_pass(StepArgs A) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= A.N) return;
  if (blockIdx.y == 0) bond_pass_axis<0>(A, v);
  else if (blockIdx.y == 1) bond_pass_axis<1>(A, v);
  else bond_pass_axis<2>(A, v);
}

// Bond sums in the fixed order +x, +y, +z (the voxel is voxel 1: F1, M1),
// then -x, -y, -z (the voxel is voxel 2: -F1, M2); both forms use it.
__global__ void __launch_bounds__(256) voxel_pass(StepArgs A) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  bool active = v < A.N;
  float speed = 0.f;
  int body = 0;
  if (active) {
    const int64_t P = A.pitch, C = 3 * P;
    const VoxMeta mt = load_meta(A, v);
    body = mt.b;
    V3f F = v3(0.f, 0.f, 0.f), M = v3(0.f, 0.f, 0.f);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (A.nbr[(int64_t)(2 * a + 1) * A.N + v] >= 0) {
        const float* bf = A.bf + (int64_t)a * P + v;
        F = add(F, v3(bf[0], bf[C], bf[2 * C]));
        M = add(M, v3(bf[3 * C], bf[4 * C], bf[5 * C]));
      }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      int un = A.nbr[(int64_t)(2 * a) * A.N + v];
      if (un >= 0) {
        const float* bf = A.bf + (int64_t)a * P + un;
        F = add(F, v3(-bf[0], -bf[C], -bf[2 * C]));
        M = add(M, v3(bf[6 * C], bf[7 * C], bf[8 * C]));
      }
    }
    VoxS s = load_vox(A.st_in, P, v);
    speed = voxel_finish(A, v, mt, s, F, M, thermal_strain(A, v, A.mats[mt.m].cte), voxel_E(A, v, mt.m), A.mats);
  }
  if (A.collide_on) horizon_max(A, body, active, speed);
}

// ---------------------------------------------------------------------------
// fused form
// ---------------------------------------------------------------------------
// One CTA per tile.  Every global read the step needs is issued in the
// staging phase (independent loads, one round trip, plus one for the halo
// indices), so the bond and voxel phases run on shared memory and registers
// only and the SM overlaps one CTA's staging with the others' arithmetic.
// Shared memory, ML = 2 TMAX staged voxels (owned first, then the halo):
//   st[13][ML]                      staged state
//   E, G, adT, m, I [ML]            modulus, shear modulus, thermal strain, mass, inertia
//   slot[3 axes][6][TMAX]           result of the bond on each owned voxel's
//                                   -a side: (-F1, M2)
//   hb[ML]                          the tile's halo bonds
//   mats[n_mat]                     material table
template <int TMAX> struct FusedSmem {
  static constexpr int ML = 2 * TMAX;
  static constexpr int kFloats = (NPLANE + 6) * ML + 18 * TMAX;
  static size_t bytes(int n_mat) { return kFloats * sizeof(float) + (size_t)n_mat * sizeof(DevMat); }
};

template <int TMAX>
__device__ __forceinline__ VoxS smem_vox(const float* s_st, int k) {
  constexpr int ML = FusedSmem<TMAX>::ML;
  VoxS v;
  v.o = v3(s_st[OX * ML + k], s_st[OY * ML + k], s_st[OZ * ML + k]);
  v.q.w = s_st[QW * ML + k]; v.q.x = s_st[QX * ML + k]; v.q.y = s_st[QY * ML + k]; v.q.z = s_st[QZ * ML + k];
  v.v = v3(s_st[VX * ML + k], s_st[VY * ML + k], s_st[VZ * ML + k]);
  v.w = v3(s_st[WX * ML + k], s_st[WY * ML + k], s_st[WZ * ML + k]);
  return v;
}

template <int TMAX, int a>
__device__ __forceinline__ void store_minus_slot(float* s_slot, int k, const BondOut& o) {
  float* sl = s_slot + a * 6 * TMAX + k;
  sl[0] = -o.F1.x; sl[TMAX] = -o.F1.y; sl[2 * TMAX] = -o.F1.z;
  sl[3 * TMAX] = o.M2.x; sl[4 * TMAX] = o.M2.y; sl[5 * TMAX] = o.M2.z;
}

template <int TMAX, int a>
__device__ __forceinline__ void halo_bond(const StepArgs& A, const float* s_st, const float* s_E, const float* s_G,
                                          const float* s_adT, const float* s_m, const float* s_I, float* s_slot,
                                          int s1, int s2) {
  VoxS v1 = smem_vox<TMAX>(s_st, s1), v2 = smem_vox<TMAX>(s_st, s2);
  M3f R1 = qmat(v1.q);
  BondOut o = bond_eval<a>(v1, R1, v2, A.l, s_E[s1], s_E[s2], s_G[s1], s_G[s2], fminf(s_m[s1], s_m[s2]),
                           fminf(s_I[s1], s_I[s2]), mul_(0.5f, add_(s_adT[s1], s_adT[s2])), A.zb);
  store_minus_slot<TMAX, a>(s_slot, s2, o);
}

// Material-dependent values of one staged voxel.
__device__ __forceinline__ void slot_props(const StepArgs& A, const DevMat& d, float ph, float le, int k,
                                           float* s_E, float* s_G, float* s_adT, float* s_m, float* s_I) {
  float E = A.logE ? expf(le) : d.E;
  s_E[k] = E;
  s_G[k] = __fmul_rn(E, d.g_ratio);
  float adT = 0.f;
  if (A.act_on) {
    float x = A.act_w + ph;
    x = __fmaf_rn(-6.28318530717958648f, rintf(__fmul_rn(x, 0.159154943091895336f)), x);
    adT = __fmul_rn(d.cte, __fmaf_rn(A.actA, __sinf(x), A.actT0));
  }
  s_adT[k] = adT;
  s_m[k] = d.m;
  s_I[k] = d.I;
}

template <int TMAX>
__global__ void __launch_bounds__(TMAX, TMAX == 512 ? 1 : (TMAX == 256 ? 3 : 6)) fused_step(StepArgs A) {
  constexpr int ML = FusedSmem<TMAX>::ML;
  extern __shared__ float smem[];
  float* s_st = smem;
  float* s_E = s_st + NPLANE * ML;
  float* s_G = s_E + ML;
  float* s_adT = s_G + ML;
  float* s_m = s_adT + ML;
  float* s_I = s_m + ML;
  float* s_slot = s_I + ML;
  uint32_t* s_hb = reinterpret_cast<uint32_t*>(s_slot + 18 * TMAX);
  DevMat* s_mats = reinterpret_cast<DevMat*>(s_hb + ML);
  const int i = threadIdx.x;
  const int4 ta = A.tile_a[blockIdx.x];
  const int4 tb = A.tile_b[blockIdx.x];
  const int v0 = ta.x, T = ta.y, NL = ta.y + ta.w, nhb = tb.y - tb.x;
  const int P = (int)A.pitch;
  const bool own = i < T;
  const int v = v0 + i;
  // ---- staging: every global read of the step, issued back to back
  const int k1 = i + TMAX;
  const int g0 = own ? v : (i < NL ? A.halo[ta.z + i - T] : -1);
  const int g1 = k1 < NL ? (k1 < T ? v0 + k1 : A.halo[ta.z + k1 - T]) : -1;
  float r0[NPLANE], r1[NPLANE];
#pragma unroll
  for (int p = 0; p < NPLANE; ++p) {
    r0[p] = g0 >= 0 ? A.st_in[g0 + p * P] : 0.f;
    r1[p] = g1 >= 0 ? A.st_in[g1 + p * P] : 0.f;
  }
  const int m0 = g0 >= 0 ? A.mat[g0] : 0, m1 = g1 >= 0 ? A.mat[g1] : 0;
  const float ph0 = (g0 >= 0 && A.phase) ? A.phase[g0] : 0.f, ph1 = (g1 >= 0 && A.phase) ? A.phase[g1] : 0.f;
  const float le0 = (g0 >= 0 && A.logE) ? A.logE[g0] : 0.f, le1 = (g1 >= 0 && A.logE) ? A.logE[g1] : 0.f;
  int px = 0xFFFF, py = 0xFFFF, pz = 0xFFFF;
  uint32_t mask = 0;
  VoxMeta mt;
  if (own) {
    px = A.plus[v]; py = A.plus[A.N + v]; pz = A.plus[2 * A.N + v];
    mask = A.mask[v];
    mt = load_meta(A, v);
  }
  for (int j = i; j < nhb; j += TMAX) s_hb[j] = A.hbonds[tb.x + j];
  for (int j = i; j < A.n_mats * (int)(sizeof(DevMat) / 4); j += TMAX)
    reinterpret_cast<float*>(s_mats)[j] = reinterpret_cast<const float*>(A.mats)[j];
#pragma unroll
  for (int p = 0; p < NPLANE; ++p) {
    if (g0 >= 0) s_st[p * ML + i] = r0[p];
    if (g1 >= 0) s_st[p * ML + k1] = r1[p];
  }
  __syncthreads();
  if (g0 >= 0) slot_props(A, s_mats[m0], ph0, le0, i, s_E, s_G, s_adT, s_m, s_I);
  if (g1 >= 0) slot_props(A, s_mats[m1], ph1, le1, k1, s_E, s_G, s_adT, s_m, s_I);
  __syncthreads();
  // ---- bonds: this voxel's own +x, +y, +z bonds, state and rotation loaded once
  V3f F = v3(0.f, 0.f, 0.f), M = v3(0.f, 0.f, 0.f);
  VoxS s;
  if (own) {
    s = smem_vox<TMAX>(s_st, i);
    M3f R1 = qmat(s.q);
    float E1 = s_E[i], G1 = s_G[i], adT1 = s_adT[i], mm1 = s_m[i], I1 = s_I[i];
#define VX_PLUS_BOND(AX, P2)                                                                               \
    if (P2 != 0xFFFF) {                                                                                    \
      VoxS v2 = smem_vox<TMAX>(s_st, P2);                                                                  \
      BondOut o = bond_eval<AX>(s, R1, v2, A.l, E1, s_E[P2], G1, s_G[P2], fminf(mm1, s_m[P2]),             \
                                fminf(I1, s_I[P2]), mul_(0.5f, add_(adT1, s_adT[P2])), A.zb);            \
      F = add(F, o.F1);                                                                                    \
      M = add(M, o.M1);                                                                                    \
      if (P2 < T) store_minus_slot<TMAX, AX>(s_slot, P2, o);                                               \
    }
    VX_PLUS_BOND(0, px)
    VX_PLUS_BOND(1, py)
    VX_PLUS_BOND(2, pz)
#undef VX_PLUS_BOND
  }
  // bonds whose negative-side voxel is in the halo
  for (int j = i; j < nhb; j += TMAX) {
    uint32_t pk = s_hb[j];
    int s1 = (int)(pk & 4095u), s2 = (int)((pk >> 12) & 4095u), ax = (int)(pk >> 24);
    if (ax == 0) halo_bond<TMAX, 0>(A, s_st, s_E, s_G, s_adT, s_m, s_I, s_slot, s1, s2);
    else if (ax == 1) halo_bond<TMAX, 1>(A, s_st, s_E, s_G, s_adT, s_m, s_I, s_slot, s1, s2);
    else halo_bond<TMAX, 2>(A, s_st, s_E, s_G, s_adT, s_m, s_I, s_slot, s1, s2);
  }
  __syncthreads();
  // ---- gather the -x, -y, -z results and integrate
  float speed = 0.f;
  if (own) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
      if (mask & (1u << (2 * a))) {
        const float* sl = s_slot + a * 6 * TMAX + i;
        F = add(F, v3(sl[0], sl[TMAX], sl[2 * TMAX]));
        M = add(M, v3(sl[3 * TMAX], sl[4 * TMAX], sl[5 * TMAX]));
      }
    speed = voxel_finish(A, v, mt, s, F, M, s_adT[i], s_E[i], s_mats);
  }
  if (A.collide_on) horizon_max(A, own ? mt.b : 0, own, speed);
}

size_t fused_smem_bytes(int tile_max, int n_mats) {
  if (tile_max == 128) return FusedSmem<128>::bytes(n_mats);
  if (tile_max == 256) return FusedSmem<256>::bytes(n_mats);
  return FusedSmem<512>::bytes(n_mats);
}

int prepare_fused(int tile_max, size_t smem) {
  cudaError_t e = cudaErrorInvalidValue;
  if (tile_max == 256) e = cudaFuncSetAttribute(fused_step<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  else if (tile_max == 128) e = cudaFuncSetAttribute(fused_step<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  else if (tile_max == 512) e = cudaFuncSetAttribute(fused_step<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return e == cudaSuccess ? 0 : -1;
}

void launch_step(const StepArgs& A, int form, int tile_max, size_t smem, cudaStream_t s) {
  if (form == 0) {
    if (tile_max == 256) fused_step<256><<<A.n_tiles, 256, smem, s>>>(A);
    else if (tile_max == 128) fused_step<128><<<A.n_tiles, 128, smem, s>>>(A);
    else fused_step<512><<<A.n_tiles, 512, smem, s>>>(A);
  } else {
    dim3 blk(256);
    bond_pass<<<dim3((A.N + 255) / 256, 3), blk, 0, s>>>(A);
    voxel_pass<<<(A.N + 255) / 256, blk, 0, s>>>(A);
  }
}

}  // namespace vx

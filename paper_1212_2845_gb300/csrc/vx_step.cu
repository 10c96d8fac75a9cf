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
  BondK k;
  if (A.lut) {
    k = lut_consts(A.lut, A.n_mats, m1, m2);
  } else {
    float E1 = voxel_E(A, v, m1), E2 = voxel_E(A, u, m2);
    k = bond_consts(A.l, E1, E2, __fmul_rn(E1, d1.g_ratio), __fmul_rn(E2, d2.g_ratio), fminf(d1.m, d2.m),
                    fminf(d1.I, d2.I), A.zb);
  }
  float eps = mul_(0.5f, add_(thermal_strain(A, v, d1), thermal_strain(A, u, d2)));
  BondOut o = bond_eval<a>(s1, qmat(s1.q), s2, A.l, k, eps, A.zb != 0.f);
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
    store_bond_sums(A, v, F, M);
    speed = voxel_finish(A, v, mt, s, F, M, thermal_strain(A, v, A.mats[mt.m]), voxel_E(A, v, mt.m), A.mats);
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
//   state: A, B, C float4 [ML], D float [ML]   (same planes as in HBM)
//   props float4 [ML]: E, G, thermal strain, material index (bits)
//   slot F4 float4 [3][TMAX], slot F2 float2 [3][TMAX]: the result of the bond
//        on each owned voxel's -a side: (-F1, M2.x) and (M2.y, M2.z)
//   hb uint32 [ML]: the tile's halo bonds
//   lut float [8 n_mats^2] (when set), mats DevMat [n_mats]
#ifndef VX_CTAS_256
#define VX_CTAS_256 3  // resident CTAs per SM of fused_step<256> (registers <= 85)
#endif

template <int TMAX> struct FusedSmem {
  static constexpr int ML = 2 * TMAX;
  static constexpr int kFloats = (NPLANE + 4 + 1) * ML + 18 * TMAX;
  static size_t bytes(int n_mats, bool lut) {
    return kFloats * sizeof(float) + (lut ? (size_t)8 * n_mats * n_mats * sizeof(float) : 0) +
           (size_t)n_mats * sizeof(DevMat);
  }
};

template <int TMAX> struct Smem {
  float4 *A, *B, *C, *props, *slotF4;
  float *D, *lut;
  float2* slotF2;
  uint32_t* hb;
  DevMat* mats;
  __device__ __forceinline__ Smem(float* base, int n_mats, bool has_lut) {
    constexpr int ML = FusedSmem<TMAX>::ML;
    A = reinterpret_cast<float4*>(base);
    B = A + ML;
    C = B + ML;
    props = C + ML;
    slotF4 = props + ML;
    slotF2 = reinterpret_cast<float2*>(slotF4 + 3 * TMAX);
    D = reinterpret_cast<float*>(slotF2 + 3 * TMAX);
    hb = reinterpret_cast<uint32_t*>(D + ML);
    lut = reinterpret_cast<float*>(hb + ML);
    mats = reinterpret_cast<DevMat*>(lut + (has_lut ? 8 * n_mats * n_mats : 0));
  }
  __device__ __forceinline__ VoxS vox(int k) const { return unpack_vox(A[k], B[k], C[k], D[k]); }
};

__device__ __forceinline__ void store_minus_slot_r(float4* F4, float2* F2, int tmax, int k, int a, const BondOut& o) {
  F4[a * tmax + k] = make_float4(-o.F1.x, -o.F1.y, -o.F1.z, o.M2.x);
  F2[a * tmax + k] = make_float2(o.M2.y, o.M2.z);
}
template <int TMAX, int a>
__device__ __forceinline__ void store_minus_slot(const Smem<TMAX>& S, int k, const BondOut& o) {
  store_minus_slot_r(S.slotF4, S.slotF2, TMAX, k, a, o);
}

// Constants of the bond between staged voxels k1 and k2.
template <int TMAX>
__device__ __forceinline__ BondK staged_consts(const StepArgs& A, const Smem<TMAX>& S, float4 p1, float4 p2) {
  int m1 = __float_as_int(p1.w), m2 = __float_as_int(p2.w);
  if (A.lut) return lut_consts(S.lut, A.n_mats, m1, m2);
  const DevMat& d1 = S.mats[m1];
  const DevMat& d2 = S.mats[m2];
  return bond_consts(A.l, p1.x, p2.x, p1.y, p2.y, fminf(d1.m, d2.m), fminf(d1.I, d2.I), A.zb);
}

// A bond entering the tile from its halo: one code path for the three axes
// (lanes of a warp holding bonds of different axes do not diverge).
template <int TMAX>
__device__ __forceinline__ void halo_bond(const StepArgs& A, const Smem<TMAX>& S, int s1, int s2, int a) {
  VoxS v1 = S.vox(s1), v2 = S.vox(s2);
  float4 p1 = S.props[s1], p2 = S.props[s2];
  BondK k = staged_consts<TMAX>(A, S, p1, p2);
  BondOut o = bond_eval_r(v1, qmat(v1.q), v2, A.l, k, mul_(0.5f, add_(p1.z, p2.z)), A.zb != 0.f, a);
  store_minus_slot_r(S.slotF4, S.slotF2, TMAX, s2, a, o);
}

// Material-dependent values of one staged voxel: E, G, thermal strain, material.
__device__ __forceinline__ float4 slot_props(const StepArgs& A, const DevMat& d, int m, float ph, float le) {
  float E = A.logE ? expf(le) : d.E;
  return make_float4(E, __fmul_rn(E, d.g_ratio), strain_of(A, d, ph), __int_as_float(m));
}

template <int TMAX>
__global__ void __launch_bounds__(TMAX, TMAX == 512 ? 1 : (TMAX == 256 ? VX_CTAS_256 : 8)) fused_step(StepArgs A) {
  extern __shared__ __align__(16) float smem[];
  const Smem<TMAX> S(smem, A.n_mats, A.lut != nullptr);
  const int i = threadIdx.x;
  const int4 ta = A.tile_a[blockIdx.x];
  const int4 tb = A.tile_b[blockIdx.x];
  const int v0 = ta.x, T = ta.y, NL = ta.y + ta.w, nhb = tb.y - tb.x;
  const bool own = i < T;
  const int v = v0 + i;
  const StPtr G(const_cast<float*>(A.st_in), A.pitch);
  // ---- staging: every global read of the step, issued back to back
  const int k1 = i + TMAX;
  const int g0 = own ? v : (i < NL ? A.halo[ta.z + i - T] : -1);
  const int g1 = k1 < NL ? (k1 < T ? v0 + k1 : A.halo[ta.z + k1 - T]) : -1;
  float4 a0, b0, c0, a1, b1, c1;
  float d0, d1;
  if (g0 >= 0) { a0 = G.A[g0]; b0 = G.B[g0]; c0 = G.C[g0]; d0 = G.D[g0]; }
  if (g1 >= 0) { a1 = G.A[g1]; b1 = G.B[g1]; c1 = G.C[g1]; d1 = G.D[g1]; }
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
  for (int j = i; j < nhb; j += TMAX) S.hb[j] = A.hbonds[tb.x + j];
  for (int j = i; j < A.n_mats * (int)(sizeof(DevMat) / 4); j += TMAX)
    reinterpret_cast<float*>(S.mats)[j] = reinterpret_cast<const float*>(A.mats)[j];
  if (A.lut)
    for (int j = i; j < 8 * A.n_mats * A.n_mats; j += TMAX) S.lut[j] = A.lut[j];
  if (g0 >= 0) { S.A[i] = a0; S.B[i] = b0; S.C[i] = c0; S.D[i] = d0; }
  if (g1 >= 0) { S.A[k1] = a1; S.B[k1] = b1; S.C[k1] = c1; S.D[k1] = d1; }
  __syncthreads();
  if (g0 >= 0) S.props[i] = slot_props(A, S.mats[m0], m0, ph0, le0);
  if (g1 >= 0) S.props[k1] = slot_props(A, S.mats[m1], m1, ph1, le1);
  __syncthreads();
  // ---- bonds: this voxel's own +x, +y, +z bonds, state and rotation loaded once
  V3f F = v3(0.f, 0.f, 0.f), M = v3(0.f, 0.f, 0.f);
  VoxS s;
  float4 pr;
  if (own) {
    s = S.vox(i);
    pr = S.props[i];
    const M3f R1 = qmat(s.q);
    const bool damp = A.zb != 0.f;
#define VX_PLUS_BOND(AX, P2)                                                                               \
    if (P2 != 0xFFFF) {                                                                                    \
      const VoxS v2 = S.vox(P2);                                                                           \
      const float4 q2 = S.props[P2];                                                                       \
      const BondK k = staged_consts<TMAX>(A, S, pr, q2);                                                   \
      BondOut o = bond_eval<AX>(s, R1, v2, A.l, k, mul_(0.5f, add_(pr.z, q2.z)), damp);                     \
      F = add(F, o.F1);                                                                                    \
      M = add(M, o.M1);                                                                                    \
      if (P2 < T) store_minus_slot<TMAX, AX>(S, P2, o);                                                    \
    }
    VX_PLUS_BOND(0, px)
    VX_PLUS_BOND(1, py)
    VX_PLUS_BOND(2, pz)
#undef VX_PLUS_BOND
  }
  // bonds whose negative-side voxel is in the halo
  for (int j = i; j < nhb; j += TMAX) {
    uint32_t pk = S.hb[j];
    int s1 = (int)(pk & 4095u), s2 = (int)((pk >> 12) & 4095u), ax = (int)(pk >> 24);
    halo_bond<TMAX>(A, S, s1, s2, ax);
  }
  __syncthreads();
  // ---- gather the -x, -y, -z results and integrate
  float speed = 0.f;
  if (own) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
      if (mask & (1u << (2 * a))) {
        const float4 f = S.slotF4[a * TMAX + i];
        const float2 g = S.slotF2[a * TMAX + i];
        F = add(F, v3(f.x, f.y, f.z));
        M = add(M, v3(f.w, g.x, g.y));
      }
    store_bond_sums(A, v, F, M);
    speed = voxel_finish(A, v, mt, s, F, M, pr.z, pr.x, S.mats);
  }
  if (A.collide_on) horizon_max(A, own ? mt.b : 0, own, speed);
}

size_t fused_smem_bytes(int tile_max, int n_mats, bool lut) {
  if (tile_max == 128) return FusedSmem<128>::bytes(n_mats, lut);
  if (tile_max == 256) return FusedSmem<256>::bytes(n_mats, lut);
  return FusedSmem<512>::bytes(n_mats, lut);
}

template <int TMAX> int prepare_one(size_t smem) {
  if (allow_smem(fused_step<TMAX>, smem) != cudaSuccess)
    return -1;
  return 0;
}

int prepare_fused(int tile_max, size_t smem) {
  if (tile_max == 256) return prepare_one<256>(smem);
  if (tile_max == 128) return prepare_one<128>(smem);
  if (tile_max == 512) return prepare_one<512>(smem);
  return -1;
}

void launch_bond_pass(const StepArgs& A, cudaStream_t s) {
  bond_pass<<<dim3((A.N + 255) / 256, 3), 256, 0, s>>>(A);
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

// Pipelined form of the fused step (same arithmetic, same bits).
//
// Persistent CTAs walk the tiles t = blockIdx.x, + gridDim.x, ...  While tile
// t is computed, everything tile t + gridDim.x needs (state of its owned and
// halo voxels, material words, bond partner slots, lattice coordinates, halo
// bonds) streams into the other half of a double-buffered shared staging area
// with cp.async, and the descriptor and halo indices of the tile after it are
// already on their way into registers.  Tile descriptors and halo index lists
// live at fixed strides so that both arrive in one round trip.
#include "vx_collide.cuh"

namespace vx {
namespace {

__device__ __forceinline__ uint32_t sptr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp16(void* d, const void* s) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sptr(d)), "l"(s) : "memory");
}
__device__ __forceinline__ void cp8(void* d, const void* s) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sptr(d)), "l"(s) : "memory");
}
__device__ __forceinline__ void cp4(void* d, const void* s) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sptr(d)), "l"(s) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Descriptor of a tile held in registers (h0, h1: halo voxels of list
// positions threadIdx.x and threadIdx.x + TMAX).
struct TileRegs {
  int v0, T, nh, hb0, nhb, h0, h1;
  bool valid;
};

template <int TMAX>
__device__ __forceinline__ TileRegs load_tile(const StepArgs& A, int t, int t_end) {
  TileRegs r;
  r.valid = t < t_end;
  if (!r.valid) { r.v0 = r.T = r.nh = r.hb0 = r.nhb = 0; r.h0 = r.h1 = -1; return r; }
  const int4 d = reinterpret_cast<const int4*>(A.tdesc)[2 * t];
  const int b0 = reinterpret_cast<const int4*>(A.tdesc)[2 * t + 1].x;
  const int32_t* hf = A.hfix + (int64_t)t * A.hstride;
  r.v0 = d.x; r.T = d.y; r.nh = d.z; r.hb0 = d.w; r.nhb = b0;
  r.h0 = hf[threadIdx.x];
  r.h1 = threadIdx.x + TMAX < A.hstride ? hf[threadIdx.x + TMAX] : -1;
  return r;
}

// Staging buffer of one tile (ML = 2 TMAX slots: owned first, then the halo).
template <int TMAX> struct Stage {
  static constexpr int ML = 2 * TMAX;
  float4 *A, *B, *C;
  float* D;
  uint32_t* vw;    // material | bond mask << 8
  float *ph, *le;  // phase, log E (null when unused)
  uint2* pl;       // +x, +y, +z partner slots of owned voxels
  uint32_t* lat;
  int32_t* body;   // null for one body
  float* fx;       // 3 x TMAX external force (null when unused)
  int32_t* nc;     // collision candidates of owned voxels (null without collisions)
  uint32_t* hb;    // halo bonds
  // floats this layout needs
  static __host__ __device__ int floats(bool ph, bool le, bool body, bool fext, bool col) {
    return 13 * ML + ML + (ph ? ML : 0) + (le ? ML : 0) + 2 * TMAX + TMAX + (body ? TMAX : 0) + (fext ? 3 * TMAX : 0) +
           ML + (col ? TMAX : 0);
  }
  __device__ __forceinline__ void carve(float* base, bool hph, bool hle, bool hbody, bool hfext, bool hcol) {
    A = reinterpret_cast<float4*>(base);
    B = A + ML;
    C = B + ML;
    pl = reinterpret_cast<uint2*>(C + ML);
    float* p = reinterpret_cast<float*>(pl + TMAX);
    D = p; p += ML;
    vw = reinterpret_cast<uint32_t*>(p); p += ML;
    lat = reinterpret_cast<uint32_t*>(p); p += TMAX;
    hb = reinterpret_cast<uint32_t*>(p); p += ML;
    ph = hph ? p : nullptr; p += hph ? ML : 0;
    le = hle ? p : nullptr; p += hle ? ML : 0;
    body = hbody ? reinterpret_cast<int32_t*>(p) : nullptr; p += hbody ? TMAX : 0;
    fx = hfext ? p : nullptr; p += hfext ? 3 * TMAX : 0;
    nc = hcol ? reinterpret_cast<int32_t*>(p) : nullptr;
  }
  __device__ __forceinline__ VoxS vox(int k) const { return unpack_vox(A[k], B[k], C[k], D[k]); }
};

template <int TMAX>
__device__ __forceinline__ void stage_voxel(const StepArgs& A, const StPtr& G, const Stage<TMAX>& S, int k, int g) {
  cp16(&S.A[k], &G.A[g]);
  cp16(&S.B[k], &G.B[g]);
  cp16(&S.C[k], &G.C[g]);
  cp4(&S.D[k], &G.D[g]);
  cp4(&S.vw[k], &A.vw[g]);
  if (S.ph) cp4(&S.ph[k], &A.phase[g]);
  if (S.le) cp4(&S.le[k], &A.logE[g]);
}

template <int TMAX>
__device__ __forceinline__ void issue_tile(const StepArgs& A, const StPtr& G, const Stage<TMAX>& S, const TileRegs& r) {
  const int i = threadIdx.x;
  if (i < r.T) {
    const int g = r.v0 + i;
    stage_voxel<TMAX>(A, G, S, i, g);
    cp8(&S.pl[i], &A.plus2[g]);
    cp4(&S.lat[i], &A.lat[g]);
    if (S.body) cp4(&S.body[i], &A.body[g]);
    if (S.nc) cp4(&S.nc[i], &A.vcnt[g]);
    if (S.fx) {
      cp4(&S.fx[i], &A.fext[g]);
      cp4(&S.fx[TMAX + i], &A.fext[A.pitch + g]);
      cp4(&S.fx[2 * TMAX + i], &A.fext[2 * A.pitch + g]);
    }
  }
  if (i < r.nh && VX_IN_BOUNDS(A.status, r.h0, A.N, kSiteHalo)) stage_voxel<TMAX>(A, G, S, r.T + i, r.h0);
  if (i + TMAX < r.nh && VX_IN_BOUNDS(A.status, r.h1, A.N, kSiteHalo)) stage_voxel<TMAX>(A, G, S, r.T + i + TMAX, r.h1);
  if (i < r.nhb) cp4(&S.hb[i], &A.hbonds[r.hb0 + i]);
  if (i + TMAX < r.nhb) cp4(&S.hb[i + TMAX], &A.hbonds[r.hb0 + i + TMAX]);
}

// Result of a bond for its voxel 2 (the owner's -a bond): F1 (voxel 2
// receives -F1, subtracted at the gather) and M2.
template <int TMAX>
__device__ __forceinline__ void minus_slot_r(float4* F4, float2* F2, int k, int a, const BondOut& o) {
  F4[a * TMAX + k] = make_float4(o.F1.x, o.F1.y, o.F1.z, o.M2.x);
  F2[a * TMAX + k] = make_float2(o.M2.y, o.M2.z);
}
template <int TMAX, int a>
__device__ __forceinline__ void minus_slot(float4* F4, float2* F2, int k, const BondOut& o) {
  minus_slot_r<TMAX>(F4, F2, k, a, o);
}

__device__ __forceinline__ BondK pair_consts(const StepArgs& A, const float* lut, const DevMat* mats, float4 p1,
                                             float4 p2) {
  int m1 = __float_as_int(p1.w), m2 = __float_as_int(p2.w);
  if (A.lut) return lut_consts(lut, A.n_mats, m1, m2);
  return bond_consts(A.l, p1.x, p2.x, p1.y, p2.y, fminf(mats[m1].m, mats[m2].m), fminf(mats[m1].I, mats[m2].I), A.zb);
}

__device__ __forceinline__ float4 voxel_props(const StepArgs& A, const DevMat& d, int m, float ph, float le) {
  float E = A.logE ? expf(le) : d.E;
  return make_float4(E, __fmul_rn(E, d.g_ratio), strain_of(A, d, ph), __int_as_float(m));
}

// A bond entering the tile from its halo (voxel 1 in the halo, voxel 2
// owned): one code path for the three axes, the axis a register value.
template <int TMAX>
__device__ __forceinline__ void halo_bond_p(const StepArgs& A, const Stage<TMAX>& S, const float4* props,
                                            const float* lut, const DevMat* mats, float4* F4, float2* F2, int s1,
                                            int s2, int a) {
  VoxS v1 = S.vox(s1), v2 = S.vox(s2);
  float4 p1 = props[s1], p2 = props[s2];
  BondK k = pair_consts(A, lut, mats, p1, p2);
  BondOut o = bond_eval_r(v1, qmat(v1.q), v2, A.l, k, mul_(0.5f, add_(p1.z, p2.z)), A.zb != 0.f, a);
  minus_slot_r<TMAX>(F4, F2, s2, a, o);
}

// Material properties (E, G, thermal strain, material) of the slots this
// thread staged itself (owned voxel i, halo list positions i and i + TMAX):
// after its own copies have landed they need no barrier.
template <int TMAX>
__device__ __forceinline__ void tile_props(const StepArgs& A, const Stage<TMAX>& S, float4* props,
                                           const DevMat* mats, const TileRegs& r) {
  const int i = threadIdx.x;
  if (i < r.T) {
    const uint32_t w = S.vw[i];
    props[i] = voxel_props(A, mats[w & 255u], (int)(w & 255u), S.ph ? S.ph[i] : 0.f, S.le ? S.le[i] : 0.f);
  }
  for (int j = i; j < r.nh; j += TMAX) {
    const int k = r.T + j;
    const uint32_t w = S.vw[k];
    props[k] = voxel_props(A, mats[w & 255u], (int)(w & 255u), S.ph ? S.ph[k] : 0.f, S.le ? S.le[k] : 0.f);
  }
}

// Everything after a tile's staging and properties are in place: own and
// halo bonds, gather and the voxel update.  Between the bond results and the
// gather (after the barrier that publishes the results, when nobody reads
// the property slots any more) the thread waits for its copies of the next
// tile and writes that tile's properties.
template <int TMAX>
__device__ __forceinline__ void compute_tile(const StepArgs& A, const Stage<TMAX>& S, float4* props, float4* F4,
                                             float2* F2, const DevMat* mats, const float* lut, const TileRegs& cur,
                                             uint8_t fl_cur, const Stage<TMAX>& Sn, const TileRegs& nxt,
                                             float& vrun) {
  const int i = threadIdx.x;
  const int T = cur.T;
  const bool own = i < T;
  // own +x, +y, +z bonds; halo bonds
  V3f F = v3(0.f, 0.f, 0.f), M = v3(0.f, 0.f, 0.f);
  VoxS s;
  float4 pr;
  uint32_t w0 = 0;
  if (own) {
    s = S.vox(i);
    pr = props[i];
    w0 = S.vw[i];
    const uint2 pl = S.pl[i];
    const int px = (int)(pl.x & 0xFFFFu), py = (int)(pl.x >> 16), pz = (int)(pl.y & 0xFFFFu);
    const M3f R1 = qmat(s.q);
    const bool damp = A.zb != 0.f;
#define VX_PLUS_BOND(AX, P2)                                                                               \
    if (P2 != 0xFFFF && VX_IN_BOUNDS(A.status, P2, T + cur.nh, kSitePlusSlot)) {                         \
      const VoxS v2 = S.vox(P2);                                                                         \
      const float4 q2 = props[P2];                                                                       \
      const BondK k = pair_consts(A, lut, mats, pr, q2);                                                 \
      BondOut o = bond_eval<AX>(s, R1, v2, A.l, k, mul_(0.5f, add_(pr.z, q2.z)), damp);                   \
      F = add(F, o.F1);                                                                                  \
      M = add(M, o.M1);                                                                                  \
      if (P2 < T) minus_slot<TMAX, AX>(F4, F2, P2, o);                                                   \
    }
    VX_PLUS_BOND(0, px)
    VX_PLUS_BOND(1, py)
    VX_PLUS_BOND(2, pz)
#undef VX_PLUS_BOND
  }
  for (int j = i; j < cur.nhb; j += TMAX) {
    const uint32_t pk = S.hb[j];
    const int s1 = (int)(pk & 4095u), s2 = (int)((pk >> 12) & 4095u), ax = (int)(pk >> 24);
    if (!VX_IN_BOUNDS(A.status, s1, T + cur.nh, kSiteHaloBond) || !VX_IN_BOUNDS(A.status, s2, T, kSiteHaloBond) ||
        !VX_IN_BOUNDS(A.status, ax, 3, kSiteHaloBond))
      continue;
    halo_bond_p<TMAX>(A, S, props, lut, mats, F4, F2, s1, s2, ax);
  }
  __syncthreads();
  if (nxt.valid) {
    cp_wait_all();
    tile_props<TMAX>(A, Sn, props, mats, nxt);
  }
  // gather the -x, -y, -z results and integrate
  float speed = 0.f;
  int body = 0;
  if (own) {
    const uint32_t mask = (w0 >> 8) & 63u;
#pragma unroll
    for (int a = 0; a < 3; ++a)
      if (mask & (1u << (2 * a))) {
        const float4 f = F4[a * TMAX + i];
        const float2 g = F2[a * TMAX + i];
        F = sub(F, v3(f.x, f.y, f.z));  // F - F1 is F + (-F1) exactly
        M = add(M, v3(f.w, g.x, g.y));
      }
    VoxMeta mt;
    mt.lat = S.lat[i];
    mt.m = (int)(w0 & 255u);
    mt.b = S.body ? S.body[i] : 0;
    mt.fl = fl_cur;
    mt.dt = A.dt_body[mt.b];
    mt.z0 = fma_(add_((float)(int)(mt.lat >> 22), 0.5f), A.l, A.origin[3 * mt.b + 2]);
    mt.fext = S.fx ? v3(S.fx[i], S.fx[TMAX + i], S.fx[2 * TMAX + i]) : v3(0.f, 0.f, 0.f);
    mt.nc = S.nc ? S.nc[i] : 0;
    body = mt.b;
    store_bond_sums(A, cur.v0 + i, F, M);
    speed = voxel_finish(A, cur.v0 + i, mt, s, F, M, pr.z, pr.x, mats);
  }
  // the collision horizon's largest speed: per tile when the tiles of a CTA
  // may belong to several bodies, else kept in a register over all tiles
  if (A.collide_on) {
    if (A.body) horizon_max(A, body, own, speed);
    else if (own) vrun = fmaxf(vrun, speed);
  }
}

// One step over the tiles t, t + stride, ... < t_end (pipelined staging; two
// CTA barriers per tile).  Each pass of the loop starts at a barrier that
// publishes tile t (staged, properties written) and frees the other staging
// buffer and the shared bond results of tile t - stride; the copies of the
// next tile are issued right after it and land while tile t is computed.
// Ends with no copy in flight; the caller separates two calls with a
// barrier because the shared buffers are reused.
template <int TMAX>
__device__ __forceinline__ void pipe_tiles(const StepArgs& A, int t, int stride, int t_end, float* smem, int sf,
                                           float4* props, float4* F4, float2* F2, const DevMat* mats,
                                           const float* lut) {
  const bool hph = A.phase != nullptr, hle = A.logE != nullptr, hbody = A.body != nullptr, hfx = A.fext != nullptr;
  const bool hcol = A.collide_on != 0;
  const int i = threadIdx.x;
  const StPtr G(const_cast<float*>(A.st_in), A.pitch);
  // prologue: stage the first tile and write its properties
  TileRegs cur = load_tile<TMAX>(A, t, t_end);
  {
    Stage<TMAX> S0;
    S0.carve(smem, hph, hle, hbody, hfx, hcol);
    issue_tile<TMAX>(A, G, S0, cur);
    cp_commit();
    cp_wait_all();
    tile_props<TMAX>(A, S0, props, mats, cur);
  }
  uint8_t fl_cur = i < cur.T ? A.flags[cur.v0 + i] : 0;
  TileRegs nxt = load_tile<TMAX>(A, t + stride, t_end);
  int b = 0;
  float vrun = 0.f;  // largest speed of this thread's voxels (one body)
  for (;;) {
    Stage<TMAX> S, Sn;
    S.carve(smem + b * sf, hph, hle, hbody, hfx, hcol);
    Sn.carve(smem + (b ^ 1) * sf, hph, hle, hbody, hfx, hcol);
    __syncthreads();
    // stream the next tile into the other buffer, its flags into a register
    uint8_t fl_nxt = 0;
    if (nxt.valid) {
      issue_tile<TMAX>(A, G, Sn, nxt);
      cp_commit();
      fl_nxt = i < nxt.T ? A.flags[nxt.v0 + i] : 0;
    }
    // descriptor and halo indices of the tile after it
    const TileRegs nn = load_tile<TMAX>(A, t + 2 * stride, t_end);
    compute_tile<TMAX>(A, S, props, F4, F2, mats, lut, cur, fl_cur, Sn, nxt, vrun);
    if (!nxt.valid) break;  // uniform
    cur = nxt;
    nxt = nn;
    fl_cur = fl_nxt;
    t += stride;
    b ^= 1;
  }
  if (hcol && !hbody) horizon_max(A, 0, true, vrun);  // one atomic per warp for all its tiles
}

}  // namespace

template <int TMAX> struct PipeSmem {
  static constexpr int ML = 2 * TMAX;
  static size_t bytes(bool ph, bool le, bool body, bool fext, bool col, int n_mats, bool lut) {
    size_t f = 2 * (size_t)Stage<TMAX>::floats(ph, le, body, fext, col) + 4 * ML + 18 * TMAX;
    return f * sizeof(float) + (size_t)n_mats * sizeof(DevMat) + (lut ? (size_t)8 * n_mats * n_mats * 4 : 0);
  }
};

template <int TMAX> struct PipeLayout {
  int sf;
  float4 *props, *F4;
  float2* F2;
  DevMat* mats;
  float* lut;
  __device__ __forceinline__ PipeLayout(float* smem, const StepArgs& A) {
    constexpr int ML = 2 * TMAX;
    sf = Stage<TMAX>::floats(A.phase != nullptr, A.logE != nullptr, A.body != nullptr, A.fext != nullptr,
                             A.collide_on != 0);
    props = reinterpret_cast<float4*>(smem + 2 * sf);
    F4 = props + ML;
    F2 = reinterpret_cast<float2*>(F4 + 3 * TMAX);
    mats = reinterpret_cast<DevMat*>(F2 + 3 * TMAX);
    lut = reinterpret_cast<float*>(mats + A.n_mats);
  }
  __device__ __forceinline__ void load_tables(const StepArgs& A) const {
    for (int j = threadIdx.x; j < A.n_mats * (int)(sizeof(DevMat) / 4); j += TMAX)
      reinterpret_cast<float*>(mats)[j] = reinterpret_cast<const float*>(A.mats)[j];
    if (A.lut)
      for (int j = threadIdx.x; j < 8 * A.n_mats * A.n_mats; j += TMAX) lut[j] = A.lut[j];
  }
};

// LEAN > 0: a lattice without per-voxel moduli, external forces or recorded
// bond sums, whose material-pair constants come from the table (at most 16
// materials), either without actuation and per-voxel phases or with both;
// LEAN - 1 has bit 0 set for voxel contacts, bit 1 for several bodies and
// bit 2 for actuation with per-voxel phases.  Those features are then
// compile-time constants, which takes their tests and the registers they
// hold out of the per-voxel path; the arithmetic and its bits are the
// generic kernel's.
template <int TMAX, int LEAN>
__device__ __forceinline__ StepArgs lean_args(const StepArgs& A_in) {
  StepArgs A = A_in;
  if (LEAN) {
    A.act_on = ((LEAN - 1) & 4) ? 1 : 0;
    A.logE = nullptr;
    if (!((LEAN - 1) & 4)) A.phase = nullptr;
    A.fext = nullptr;
    A.fm_out = nullptr;
    if (!((LEAN - 1) & 2)) A.body = nullptr;
    A.collide_on = ((LEAN - 1) & 1) ? 1 : 0;
  }
  return A;
}

template <int TMAX, int LEAN = 0>
__global__ void __launch_bounds__(TMAX, TMAX == 128 ? 4 : (TMAX == 256 ? 2 : 1)) fused_pipe(StepArgs A_in) {
  const StepArgs A = lean_args<TMAX, LEAN>(A_in);
  if (LEAN) __builtin_assume(A.lut != nullptr);  // lean launches carry the material-pair table
  if (LEAN && ((LEAN - 1) & 4)) __builtin_assume(A.phase != nullptr);
  extern __shared__ __align__(16) float smem[];
  const PipeLayout<TMAX> L(smem, A);
  if ((int)blockIdx.x < A.n_tiles) {  // uniform over the CTA
    L.load_tables(A);
    pipe_tiles<TMAX>(A, blockIdx.x, gridDim.x, A.n_tiles, smem, L.sf, L.props, L.F4, L.F2, L.mats, L.lut);
  }
  if (A.h_done) horizon_tail(A, reinterpret_cast<float*>(L.props));
}

// Multi-step form: one cooperative launch runs n steps of the whole lattice;
// every CTA walks its tiles of a step (as fused_pipe), then all CTAs meet at
// a grid barrier before the next step reads what this one wrote.  The
// lattice stays in L2 between steps and no launch separates them.
template <int TMAX, int LEAN = 0>
__global__ void __launch_bounds__(TMAX, TMAX == 128 ? 4 : (TMAX == 256 ? 2 : 1)) multi_pipe(StepArgs A0_in, MultiArgs M) {
  const StepArgs A0 = lean_args<TMAX, LEAN>(A0_in);  // LEAN as for fused_pipe
  if (LEAN) __builtin_assume(A0.lut != nullptr);
  if (LEAN && ((LEAN - 1) & 4)) __builtin_assume(A0.phase != nullptr);
  extern __shared__ __align__(16) float smem[];
  const PipeLayout<TMAX> L(smem, A0);
  L.load_tables(A0);
  const int64_t step0 = M.ctr ? M.ctr[0] : M.step0;
  const int cur0 = M.ctr ? (int)M.ctr[1] : M.cur0;
  __syncthreads();
  for (int k = 0; k < M.n_steps; ++k) {
    StepArgs A = A0;
    const int p = (cur0 + k) & 1;
    A.st_in = p ? M.buf1 : M.buf0;
    A.st_out = p ? M.buf0 : M.buf1;
    A.step = step0 + k;
    if (A.act_on && M.act_P > 0)
      A.act_w = act_angle(A.step, M.act_P, M.act_c);
    pipe_tiles<TMAX>(A, blockIdx.x, gridDim.x, A.n_tiles, smem, L.sf, L.props, L.F4, L.F2, L.mats, L.lut);
    if (M.collide) {
      // every CTA's speeds and new state are in: horizon (or a forced
      // rebuild), then the rebuild phases when a body is flagged
      const unsigned G = gridDim.x + M.extra;
      if (!grid_barrier(M.bar, G, M.spins, A0.status)) return;
      if (blockIdx.x == 0) {
        if (M.every_step) {
          for (int b = threadIdx.x; b < A.n_bodies; b += blockDim.x) {
            A.h_flag[b] = 1;
            A.h_acc[b] = 0.f;
            A.vmax_bits[b] = 0u;
          }
          if (threadIdx.x == 0) *A.h_any = 1;
        } else {
          horizon_account(A, reinterpret_cast<float*>(L.props));
        }
      }
      if (!grid_barrier(M.bar, G, M.spins, A0.status)) return;
      if (__ldcg(A.h_any)) {  // the same value for every CTA until the last phase clears it
        CollideArgs C = M.coll;
        C.st = A.st_out;
        // the staging buffers are free between steps: the query's workspace
        if (!rebuild_phases(C, G, reinterpret_cast<int*>(smem))) return;
      }
    }
    if (k + 1 < M.n_steps && !grid_barrier(M.bar, gridDim.x + M.extra, M.spins, A0.status)) return;
  }
}

// Batched form: each CTA takes its groups of bodies one after the other and
// runs all n_steps of a group before the next; steps are separated by a CTA
// barrier, so a group's double-buffered state stays in L2 for the whole run.
// Within a step the tiles of the group are pipelined as in fused_pipe; the
// pipeline restarts after each barrier because the next step reads what this
// one wrote.
template <int TMAX, int LEAN = 0>
__global__ void __launch_bounds__(TMAX, TMAX == 128 ? 4 : (TMAX == 256 ? 2 : 1)) batched_pipe(StepArgs A0_in, BatchArgs Bt) {
  const StepArgs A0 = lean_args<TMAX, LEAN>(A0_in);  // LEAN as for fused_pipe
  if (LEAN) __builtin_assume(A0.lut != nullptr);
  if (LEAN && ((LEAN - 1) & 4)) __builtin_assume(A0.phase != nullptr);
  constexpr int ML = 2 * TMAX;
  extern __shared__ __align__(16) float smem[];
  const bool hph = A0.phase != nullptr, hle = A0.logE != nullptr, hbody = A0.body != nullptr,
             hfx = A0.fext != nullptr, hcol = A0.collide_on != 0;
  const int sf = Stage<TMAX>::floats(hph, hle, hbody, hfx, hcol);
  float4* props = reinterpret_cast<float4*>(smem + 2 * sf);
  float4* F4 = props + ML;
  float2* F2 = reinterpret_cast<float2*>(F4 + 3 * TMAX);
  DevMat* mats = reinterpret_cast<DevMat*>(F2 + 3 * TMAX);
  float* lut = reinterpret_cast<float*>(mats + A0.n_mats);
  const int i = threadIdx.x;
  for (int j = i; j < A0.n_mats * (int)(sizeof(DevMat) / 4); j += TMAX)
    reinterpret_cast<float*>(mats)[j] = reinterpret_cast<const float*>(A0.mats)[j];
  if (A0.lut)
    for (int j = i; j < 8 * A0.n_mats * A0.n_mats; j += TMAX) lut[j] = A0.lut[j];
  // first step and buffer: kernel arguments, or a device counter (graph replays)
  const int64_t step0 = Bt.ctr ? Bt.ctr[0] : Bt.step0;
  const int cur0 = Bt.ctr ? (int)Bt.ctr[1] : Bt.cur0;
  __syncthreads();
  for (int gi = Bt.cta_start[blockIdx.x]; gi < Bt.cta_start[blockIdx.x + 1]; ++gi) {
    const int g = Bt.cta_groups[gi];
    const int t0 = Bt.group_tiles[2 * g], t1 = Bt.group_tiles[2 * g + 1];
    for (int k = 0; k < Bt.n_steps; ++k) {
      StepArgs A = A0;
      const int p = (cur0 + k) & 1;
      A.st_in = p ? Bt.buf1 : Bt.buf0;
      A.st_out = p ? Bt.buf0 : Bt.buf1;
      A.step = step0 + k;
      if (A.act_on && Bt.act_P > 0)
        A.act_w = act_angle(A.step, Bt.act_P, Bt.act_c);
      pipe_tiles<TMAX>(A, t0, 1, t1, smem, sf, props, F4, F2, mats, lut);
      __syncthreads();  // the buffers are reused; the next step reads what this one wrote
    }
  }
}

size_t pipe_smem_bytes(int tile_max, bool ph, bool le, bool body, bool fext, bool col, int n_mats, bool lut) {
  if (tile_max == 128) return PipeSmem<128>::bytes(ph, le, body, fext, col, n_mats, lut);
  if (tile_max == 512) return PipeSmem<512>::bytes(ph, le, body, fext, col, n_mats, lut);
  return PipeSmem<256>::bytes(ph, le, body, fext, col, n_mats, lut);
}

namespace {

// CTAs of `kernel` (TMAX threads, smem bytes) resident on the whole device.
template <int TMAX, class K> int resident_ctas(K* kernel, size_t smem, int* n) {
  int per_sm = 0, dev = 0, n_sm = 0;
  cudaError_t e = allow_smem(kernel, smem);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, TMAX, smem);
  if (e != cudaSuccess || per_sm < 1) return -1;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return -1;
  *n = per_sm * n_sm;
  return 0;
}

// The lean variant of the 256-voxel kernel where the lattice's features
// allow it (0: the generic kernel).
static int lean_mode(const StepArgs& A) {
  if (A.logE || A.fext || A.fm_out || !A.lut || (A.act_on != 0) != (A.phase != nullptr)) return 0;
  return 1 + (A.collide_on ? 1 : 0) + (A.body ? 2 : 0) + (A.act_on ? 4 : 0);
}

template <int TMAX> int prepare_pipe_t(size_t smem, int* grid) {
  if (TMAX == 256)  // the lean variants share the generic kernel's shared memory and grid
    if (allow_smem(fused_pipe<256, 1>, smem) != cudaSuccess || allow_smem(fused_pipe<256, 2>, smem) != cudaSuccess ||
        allow_smem(fused_pipe<256, 3>, smem) != cudaSuccess || allow_smem(fused_pipe<256, 4>, smem) != cudaSuccess ||
        allow_smem(fused_pipe<256, 5>, smem) != cudaSuccess || allow_smem(fused_pipe<256, 6>, smem) != cudaSuccess ||
        allow_smem(fused_pipe<256, 7>, smem) != cudaSuccess || allow_smem(fused_pipe<256, 8>, smem) != cudaSuccess)
      return -1;
  return resident_ctas<TMAX>(fused_pipe<TMAX>, smem, grid);
}

template <int TMAX> int prepare_multi_t(size_t smem, int n_tiles, int* grid, int* co_resident) {
  int co = 0;
  if (TMAX == 256)  // the lean variants: the generic kernel's shared memory and grid (they fit it)
    if (allow_smem(multi_pipe<256, 1>, smem) != cudaSuccess || allow_smem(multi_pipe<256, 2>, smem) != cudaSuccess ||
        allow_smem(multi_pipe<256, 3>, smem) != cudaSuccess || allow_smem(multi_pipe<256, 4>, smem) != cudaSuccess ||
        allow_smem(multi_pipe<256, 5>, smem) != cudaSuccess || allow_smem(multi_pipe<256, 6>, smem) != cudaSuccess ||
        allow_smem(multi_pipe<256, 7>, smem) != cudaSuccess || allow_smem(multi_pipe<256, 8>, smem) != cudaSuccess)
      return -1;
  if (resident_ctas<TMAX>(multi_pipe<TMAX>, smem, &co) != 0) return -1;
  *grid = n_tiles < co ? n_tiles : co;
  *co_resident = co;
  return 0;
}

}  // namespace

int prepare_pipe(int tile_max, size_t smem, int* grid) {
  if (tile_max == 128) return prepare_pipe_t<128>(smem, grid);
  if (tile_max == 512) return prepare_pipe_t<512>(smem, grid);
  return prepare_pipe_t<256>(smem, grid);
}

int prepare_batched(int tile_max, size_t smem) {
  cudaError_t e;
  if (tile_max == 128) e = allow_smem(batched_pipe<128>, smem);
  else if (tile_max == 512) e = allow_smem(batched_pipe<512>, smem);
  else {
    e = allow_smem(batched_pipe<256>, smem);
    if (e == cudaSuccess) e = allow_smem(batched_pipe<256, 3>, smem);
    if (e == cudaSuccess) e = allow_smem(batched_pipe<256, 7>, smem);
  }
  return e == cudaSuccess ? 0 : -1;
}

// Batched groups are several bodies without voxel contacts: the lean
// instantiations for bodies without, and with actuation and phases.
void launch_batched(const StepArgs& A, const BatchArgs& B, int tile_max, size_t smem, int grid, cudaStream_t s) {
  if (tile_max == 128) batched_pipe<128><<<grid, 128, smem, s>>>(A, B);
  else if (tile_max == 512) batched_pipe<512><<<grid, 512, smem, s>>>(A, B);
  else switch (lean_mode(A)) {
    case 3: batched_pipe<256, 3><<<grid, 256, smem, s>>>(A, B); break;
    case 7: batched_pipe<256, 7><<<grid, 256, smem, s>>>(A, B); break;
    default: batched_pipe<256><<<grid, 256, smem, s>>>(A, B);
  }
}

int prepare_multi(int tile_max, size_t smem, int n_tiles, int* grid, int* co_resident) {
  if (tile_max == 128) return prepare_multi_t<128>(smem, n_tiles, grid, co_resident);
  if (tile_max == 512) return prepare_multi_t<512>(smem, n_tiles, grid, co_resident);
  return prepare_multi_t<256>(smem, n_tiles, grid, co_resident);
}

cudaError_t launch_multi(const StepArgs& A, const MultiArgs& M, int tile_max, size_t smem, int grid, cudaStream_t s) {
  void* args[2] = {const_cast<StepArgs*>(&A), const_cast<MultiArgs*>(&M)};
  if (tile_max == 128)
    return cudaLaunchCooperativeKernel((const void*)multi_pipe<128>, dim3(grid), dim3(128), args, smem, s);
  if (tile_max == 512)
    return cudaLaunchCooperativeKernel((const void*)multi_pipe<512>, dim3(grid), dim3(512), args, smem, s);
  const void* k = (const void*)multi_pipe<256>;
  switch (lean_mode(A)) {
    case 1: k = (const void*)multi_pipe<256, 1>; break;
    case 2: k = (const void*)multi_pipe<256, 2>; break;
    case 3: k = (const void*)multi_pipe<256, 3>; break;
    case 4: k = (const void*)multi_pipe<256, 4>; break;
    case 5: k = (const void*)multi_pipe<256, 5>; break;
    case 6: k = (const void*)multi_pipe<256, 6>; break;
    case 7: k = (const void*)multi_pipe<256, 7>; break;
    case 8: k = (const void*)multi_pipe<256, 8>; break;
    default: break;
  }
  return cudaLaunchCooperativeKernel(k, dim3(grid), dim3(256), args, smem, s);
}


void launch_pipe(const StepArgs& A, int tile_max, size_t smem, int grid, cudaStream_t s) {
  int g = grid < A.n_tiles ? grid : A.n_tiles;
  if (tile_max == 128) fused_pipe<128><<<g, 128, smem, s>>>(A);
  else if (tile_max == 512) fused_pipe<512><<<g, 512, smem, s>>>(A);
  else switch (lean_mode(A)) {
    case 1: fused_pipe<256, 1><<<g, 256, smem, s>>>(A); break;
    case 2: fused_pipe<256, 2><<<g, 256, smem, s>>>(A); break;
    case 3: fused_pipe<256, 3><<<g, 256, smem, s>>>(A); break;
    case 4: fused_pipe<256, 4><<<g, 256, smem, s>>>(A); break;
    case 5: fused_pipe<256, 5><<<g, 256, smem, s>>>(A); break;
    case 6: fused_pipe<256, 6><<<g, 256, smem, s>>>(A); break;
    case 7: fused_pipe<256, 7><<<g, 256, smem, s>>>(A); break;
    case 8: fused_pipe<256, 8><<<g, 256, smem, s>>>(A); break;
    default: fused_pipe<256><<<g, 256, smem, s>>>(A);
  }
}

}  // namespace vx

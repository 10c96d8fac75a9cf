// Plain two-pass step: per-bond kernel, then per-voxel gather + integrate.
//
// bond_pass:  one thread per (voxel, +axis) bond; writes F1, M1, M2
//             (9 floats) into bf[component][axis][voxel-1].
// voxel_pass: one thread per voxel; sums its six bond slots in the fixed
//             order -x,+x,-y,+y,-z,+z (atomic-free, deterministic), adds
//             external force, gravity, ground damping, voxel contacts and
//             floor contact with Coulomb friction, then integrates
//             (Sec 2.1.3) in place.
#include "vx_dev.cuh"
#include "vx_kernels.h"

namespace vx {

__global__ void __launch_bounds__(256) bond_pass(StepArgs A) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  int a = blockIdx.y;
  if (v >= A.N) return;
  int u = A.nbr[(int64_t)(2 * a + 1) * A.N + v];
  if (u < 0) return;
  const int64_t P = A.pitch;
  VoxS s1 = load_vox(A.st, P, v), s2 = load_vox(A.st, P, u);
  int m1 = A.mat[v], m2 = A.mat[u];
  const DevMat& d1 = A.mats[m1];
  const DevMat& d2 = A.mats[m2];
  float E1 = voxel_E(A, v, m1), E2 = voxel_E(A, u, m2);
  float eps = 0.f;
  if (A.actP > 0 || A.actT0 != 0.f)
    eps = 0.5f * (d1.cte * delta_T(A, v) + d2.cte * delta_T(A, u));
  BondOut o = bond_eval(a, s1, s2, A.l, E1, E2, E1 * d1.g_ratio, E2 * d2.g_ratio,
                        fminf(d1.m, d2.m), fminf(d1.I, d2.I), eps, A.zb);
  float* bf = A.bf + (int64_t)a * P + v;
  const int64_t C = 3 * P;  // stride between components
  bf[0 * C] = o.F1.x; bf[1 * C] = o.F1.y; bf[2 * C] = o.F1.z;
  bf[3 * C] = o.M1.x; bf[4 * C] = o.M1.y; bf[5 * C] = o.M1.z;
  bf[6 * C] = o.M2.x; bf[7 * C] = o.M2.y; bf[8 * C] = o.M2.z;
}

__device__ __forceinline__ void record_bad(const StepArgs& A, int v) {
  if (atomicOr(&A.status[0], kStatusUnstable) & kStatusUnstable) return;
  A.status[1] = v;
  *reinterpret_cast<long long*>(&A.status[2]) = (long long)A.step;
}

__global__ void __launch_bounds__(256) voxel_pass(StepArgs A) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  bool active = v < A.N;
  float speed = 0.f;
  int b = 0;
  if (active) {
    b = A.body ? A.body[v] : 0;
    uint8_t fl = A.flags[v];
    if (!(fl & 1u)) {
      const int64_t P = A.pitch, C = 3 * P;
      float* st = A.st;
      int m = A.mat[v];
      const DevMat& d = A.mats[m];
      float dt = A.dt_body[b];
      V3f F = v3(0.f, 0.f, 0.f), M = v3(0.f, 0.f, 0.f);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        int un = A.nbr[(int64_t)(2 * a) * A.N + v];
        if (un >= 0) {  // v is voxel 2 of the bond (un, v): force -F1, moment M2
          const float* bf = A.bf + (int64_t)a * P + un;
          F = sub(F, v3(bf[0], bf[C], bf[2 * C]));
          M = add(M, v3(bf[6 * C], bf[7 * C], bf[8 * C]));
        }
        int up = A.nbr[(int64_t)(2 * a + 1) * A.N + v];
        if (up >= 0) {  // v is voxel 1 of the bond (v, up): force F1, moment M1
          const float* bf = A.bf + (int64_t)a * P + v;
          F = add(F, v3(bf[0], bf[C], bf[2 * C]));
          M = add(M, v3(bf[3 * C], bf[4 * C], bf[5 * C]));
        }
      }
      if (A.fext) F = add(F, v3(A.fext[v], A.fext[P + v], A.fext[2 * P + v]));
      F.z += d.m * A.gz;
      VoxS s = load_vox(st, P, v);
      float Ev = voxel_E(A, v, m);
      float kv = Ev * A.l;
      if (A.zg != 0.f) {
        F = sub(F, scl(s.v, 2.f * A.zg * sqrtf(d.m * kv)));
        M = sub(M, scl(s.w, 2.f * A.zg * sqrtf(d.I * kv * A.l * A.l * (1.f / 6.f))));
      }
      float dT = (A.actP > 0 || A.actT0 != 0.f) ? delta_T(A, v) : 0.f;
      float h = 0.5f * A.l * (1.f + d.cte * dT);
      uint32_t lp = A.lat[v];
      int vi = (int)(lp & 2047u), vj = (int)((lp >> 11) & 2047u), vk = (int)(lp >> 22);
      if (A.collide_on) {
        int si = A.sidx[v];
        if (si >= 0) {
          int nc = A.ccount[si];
          const int32_t* cl = A.cand + (int64_t)si * kCandCap;
          for (int c = 0; c < nc; ++c) {
            int j = cl[c];
            uint32_t lq = A.lat[j];
            int dj = (int)(lq & 2047u) - vi, dk = (int)((lq >> 11) & 2047u) - vj, dl = (int)(lq >> 22) - vk;
            V3f dd = v3((float)dj * A.l + (st[OX * P + j] - s.o.x), (float)dk * A.l + (st[OY * P + j] - s.o.y),
                        (float)dl * A.l + (st[OZ * P + j] - s.o.z));
            float r = sqrtf(dot3(dd, dd));
            int mj = A.mat[j];
            const DevMat& dj_ = A.mats[mj];
            float hj = 0.5f * A.l * (1.f + dj_.cte * ((A.actP > 0 || A.actT0 != 0.f) ? delta_T(A, j) : 0.f));
            float cdist = h + hj;
            if (!(r < cdist)) continue;
            V3f nh = scl(dd, 1.f / r);
            float Ej = voxel_E(A, j, mj);
            float kc = 2.f * Ev * Ej / (Ev + Ej) * A.l;
            F = sub(F, scl(nh, kc * (cdist - r)));
            V3f vj = v3(st[VX * P + j], st[VY * P + j], st[VZ * P + j]);
            float mmin = fminf(d.m, dj_.m);
            F = add(F, scl(nh, 2.f * A.zc * sqrtf(mmin * kc) * dot3(sub(vj, s.v), nh)));
          }
        }
      }
      if (A.floor_on) {
        float z = A.origin[3 * b + 2] + ((float)vk + 0.5f) * A.l + s.o.z;
        float pen = h - z;
        if (pen > 0.f) {
          float Fn = kv * pen;
          F.z += Fn - 2.f * A.zc * sqrtf(d.m * kv) * s.v.z;
          float Flx = F.x, Fly = F.y;
          float Fl = sqrtf(Flx * Flx + Fly * Fly);
          float vl = sqrtf(s.v.x * s.v.x + s.v.y * s.v.y);
          float mus = d.mu_s * Fn, mud = d.mu_k * Fn;
          bool zero_l = false;
          if (fl & 2u) {
            if (Fl <= mus) zero_l = true;
            else { fl &= ~2u; F.x -= mud * Flx / Fl; F.y -= mud * Fly / Fl; }
          } else {
            if (vl <= mud * dt * d.inv_m && Fl <= mus) { zero_l = true; fl |= 2u; }
            else if (vl > 0.f) { F.x -= mud * s.v.x / vl; F.y -= mud * s.v.y / vl; }
            else { F.x -= mud * Flx / Fl; F.y -= mud * Fly / Fl; }
          }
          if (zero_l) { F.x = 0.f; F.y = 0.f; s.v.x = 0.f; s.v.y = 0.f; }
        } else {
          fl &= ~2u;
        }
      }
      // integrate (Sec 2.1.3): v += F/m dt; D += v dt; w += M/I dt; q <- exp(w dt) q
      float cm = dt * d.inv_m, cI = dt * d.inv_I;
      s.v = add(s.v, scl(F, cm));
      s.o = add(s.o, scl(s.v, dt));
      s.w = add(s.w, scl(M, cI));
      s.q = integrate_rot(s.q, s.w, dt);
      st[OX * P + v] = s.o.x; st[OY * P + v] = s.o.y; st[OZ * P + v] = s.o.z;
      st[QW * P + v] = s.q.w; st[QX * P + v] = s.q.x; st[QY * P + v] = s.q.y; st[QZ * P + v] = s.q.z;
      st[VX * P + v] = s.v.x; st[VY * P + v] = s.v.y; st[VZ * P + v] = s.v.z;
      st[WX * P + v] = s.w.x; st[WY * P + v] = s.w.y; st[WZ * P + v] = s.w.z;
      A.flags[v] = fl;
      float chk = s.o.x + s.o.y + s.o.z + s.v.x + s.v.y + s.v.z + s.w.x + s.w.y + s.w.z + s.q.w;
      if (!isfinite(chk)) record_bad(A, v);
      speed = sqrtf(dot3(s.v, s.v));
    }
  }
  if (A.collide_on) {
    // per-body max |v| for the collision horizon (max is order-independent)
    unsigned mask = __activemask();
    int b0 = __shfl_sync(mask, b, 0);
    bool same = __all_sync(mask, b == b0);
    if (same) {
      float s = speed;
      for (int o = 16; o > 0; o >>= 1) s = fmaxf(s, __shfl_xor_sync(mask, s, o));
      if ((threadIdx.x & 31) == 0 && s > 0.f) atomicMax(&A.vmax_bits[b0], __float_as_uint(s));
    } else if (active && speed > 0.f) {
      atomicMax(&A.vmax_bits[b], __float_as_uint(speed));
    }
  }
}

void launch_step(const StepArgs& A, cudaStream_t s) {
  dim3 blk(256);
  dim3 gb((A.N + 255) / 256, 3);
  bond_pass<<<gb, blk, 0, s>>>(A);
  voxel_pass<<<(A.N + 255) / 256, blk, 0, s>>>(A);
}

}  // namespace vx

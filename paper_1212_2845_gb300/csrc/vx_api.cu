// C ABI of the simulator (declared in include/vx.h): argument checking,
// device memory ownership and the launch sequence of each step.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "vx.h"
#include "vx_host.h"
#include "vx_kernels.h"

using namespace vx;

namespace {
thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

#define VX_CUDA(call)                                                                          \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return fail(e_ == cudaErrorMemoryAllocation ? VX_ERR_OOM : VX_ERR_CUDA,                  \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                         \
  } while (0)

template <class T> int dalloc(T** p, size_t n) {
  *p = nullptr;
  if (n == 0) n = 1;
  cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail(VX_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  return VX_OK;
}
template <class T> void dfree(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}
}  // namespace

struct vx_sim {
  Lattice L;
  int device = 0;
  int64_t pitch = 0;
  // parameters
  float zb = 1.f, zg = 0.f, zc = 1.f, gz = 0.f;
  int floor_on = 0, collide_on = 0;
  float actA = 0.f, actT0 = 0.f;
  int64_t actP = 0;
  float dt_factor = 0.9f;
  std::vector<double> dt;
  std::vector<float> logE_h;
  int64_t step = 0;
  bool has_phase = false, has_fext = false;
  // device buffers
  float* st = nullptr;
  float* bf = nullptr;
  uint8_t* flags = nullptr;
  uint8_t* mat = nullptr;
  uint32_t* lat = nullptr;
  int32_t* body = nullptr;
  int32_t* nbr = nullptr;
  float* phase = nullptr;
  float* logE = nullptr;
  float* fext = nullptr;
  DevMat* mats = nullptr;
  float* dtb = nullptr;
  float* origin = nullptr;
  int* status = nullptr;
  float* stage = nullptr;
  // collisions
  bool coll_alloc = false;
  int H = 0, qK = 0;
  int64_t qQ = 0;
  float threshold = 0.f;
  int32_t* surf = nullptr;
  int32_t* sidx = nullptr;
  int64_t* xq = nullptr;
  uint32_t* bucket = nullptr;
  uint32_t* hcount = nullptr;
  uint32_t* hcursor = nullptr;
  uint32_t* hstart = nullptr;
  uint32_t* bsum = nullptr;
  int32_t* sorted = nullptr;
  int32_t* ccount = nullptr;
  int32_t* cand = nullptr;
  float* acc = nullptr;
  unsigned* vmax = nullptr;
  int* cflag = nullptr;
  int* any = nullptr;
  long long* nreb = nullptr;
};

namespace {

StepArgs step_args(vx_sim* s) {
  StepArgs A;
  A.N = (int)s->L.N;
  A.pitch = s->pitch;
  A.l = s->L.l;
  A.st = s->st;
  A.flags = s->flags;
  A.mat = s->mat;
  A.lat = s->lat;
  A.body = s->body;
  A.nbr = s->nbr;
  A.phase = s->has_phase ? s->phase : nullptr;
  A.logE = s->logE_h.empty() ? nullptr : s->logE;
  A.fext = s->has_fext ? s->fext : nullptr;
  A.mats = s->mats;
  A.dt_body = s->dtb;
  A.origin = s->origin;
  A.bf = s->bf;
  A.zb = s->zb; A.zg = s->zg; A.zc = s->zc; A.gz = s->gz;
  A.floor_on = s->floor_on;
  A.collide_on = s->collide_on;
  A.actA = s->actA; A.actT0 = s->actT0; A.actP = s->actP;
  A.step = s->step;
  A.sidx = s->sidx;
  A.ccount = s->ccount;
  A.cand = s->cand;
  A.vmax_bits = s->vmax;
  A.status = s->status;
  return A;
}

CollideArgs collide_args(vx_sim* s) {
  CollideArgs C;
  C.S = (int)s->L.n_surface;
  C.n_bodies = s->L.n_bodies;
  C.H = s->H;
  C.K = s->qK;
  C.Q = s->qQ;
  C.pitch = s->pitch;
  C.threshold = s->threshold;
  C.st = s->st;
  C.surf = s->surf;
  C.lat = s->lat;
  C.body = s->body;
  C.dt_body = s->dtb;
  C.xq = s->xq;
  C.bucket = s->bucket;
  C.hcount = s->hcount;
  C.hcursor = s->hcursor;
  C.hstart = s->hstart;
  C.bsum = s->bsum;
  C.sorted = s->sorted;
  C.ccount = s->ccount;
  C.cand = s->cand;
  C.acc = s->acc;
  C.vmax_bits = s->vmax;
  C.flag = s->cflag;
  C.any = s->any;
  C.n_rebuilds = s->nreb;
  C.status = s->status;
  return C;
}

int upload_materials(vx_sim* s) {
  std::vector<DevMat> m(s->L.palette.size());
  double l = s->L.l;
  for (size_t i = 0; i < m.size(); ++i) {
    const vx_material& p = s->L.palette[i];
    double mass = (double)p.rho * l * l * l;
    double I = mass * l * l / 6.0;
    m[i].E = p.E;
    m[i].g_ratio = (float)(1.0 / (2.0 * (1.0 + (double)p.nu)));
    m[i].cte = p.cte;
    m[i].mu_s = p.mu_s;
    m[i].mu_k = p.mu_k;
    m[i].m = (float)mass;
    m[i].inv_m = (float)(1.0 / mass);
    m[i].I = (float)I;
    m[i].inv_I = (float)(1.0 / I);
  }
  VX_CUDA(cudaMemcpy(s->mats, m.data(), m.size() * sizeof(DevMat), cudaMemcpyHostToDevice));
  return VX_OK;
}

int upload_dt(vx_sim* s) {
  std::vector<float> f(s->dt.size());
  for (size_t b = 0; b < f.size(); ++b) f[b] = (float)s->dt[b];
  VX_CUDA(cudaMemcpy(s->dtb, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice));
  return VX_OK;
}

int recompute_dt(vx_sim* s) {
  stable_dt(s->L, s->logE_h.empty() ? nullptr : s->logE_h.data(), s->dt_factor, s->dt);
  return upload_dt(s);
}

void update_threshold(vx_sim* s) {
  double amax = 0.0;
  for (const auto& p : s->L.palette) amax = std::max(amax, (double)std::fabs(p.cte));
  double l = s->L.l;
  double cmax = l * (1.0 + amax * (std::fabs((double)s->actT0) + std::fabs((double)s->actA)));
  s->threshold = (float)(2.0 * l - cmax);
}

int alloc_collisions(vx_sim* s) {
  if (s->coll_alloc) return VX_OK;
  const Lattice& L = s->L;
  int64_t S = L.n_surface;
  int H = 1024;
  while ((int64_t)H < 2 * S) H <<= 1;
  s->H = H;
  int rc;
  if ((rc = dalloc(&s->surf, S)) || (rc = dalloc(&s->sidx, L.N)) || (rc = dalloc(&s->xq, 3 * S)) ||
      (rc = dalloc(&s->bucket, S)) || (rc = dalloc(&s->hcount, H)) || (rc = dalloc(&s->hcursor, H)) ||
      (rc = dalloc(&s->hstart, H + 1)) || (rc = dalloc(&s->bsum, (H + 1023) / 1024)) ||
      (rc = dalloc(&s->sorted, S)) || (rc = dalloc(&s->ccount, S)) || (rc = dalloc(&s->cand, S * kCandCap)) ||
      (rc = dalloc(&s->acc, L.n_bodies)) || (rc = dalloc(&s->cflag, L.n_bodies)) || (rc = dalloc(&s->any, 1)) ||
      (rc = dalloc(&s->nreb, 1)))
    return rc;
  std::vector<int32_t> sidx(L.N, -1);
  for (int64_t i = 0; i < S; ++i) sidx[L.surf_list[i]] = (int32_t)i;
  VX_CUDA(cudaMemcpy(s->surf, L.surf_list.data(), S * sizeof(int32_t), cudaMemcpyHostToDevice));
  VX_CUDA(cudaMemcpy(s->sidx, sidx.data(), L.N * sizeof(int32_t), cudaMemcpyHostToDevice));
  VX_CUDA(cudaMemset(s->ccount, 0, std::max<int64_t>(S, 1) * sizeof(int32_t)));
  VX_CUDA(cudaMemset(s->acc, 0, L.n_bodies * sizeof(float)));
  VX_CUDA(cudaMemset(s->cflag, 0, L.n_bodies * sizeof(int)));
  VX_CUDA(cudaMemset(s->any, 0, sizeof(int)));
  VX_CUDA(cudaMemset(s->nreb, 0, sizeof(long long)));
  s->coll_alloc = true;
  return VX_OK;
}

int force_rebuild(vx_sim* s, cudaStream_t st) {
  int rc = alloc_collisions(s);
  if (rc) return rc;
  update_threshold(s);
  CollideArgs C = collide_args(s);
  launch_flag_all(C, st);
  launch_rebuild(C, st);
  VX_CUDA(cudaGetLastError());
  return VX_OK;
}

int check_sim(vx_sim* s) {
  if (!s) return fail(VX_ERR_ARG, "sim is NULL");
  VX_CUDA(cudaSetDevice(s->device));
  return VX_OK;
}

int ensure_stage(vx_sim* s) {
  if (s->stage) return VX_OK;
  return dalloc(&s->stage, (size_t)14 * s->L.N);  // 13 floats + flags bytes (packed in the 14th plane)
}

}  // namespace

extern "C" {

const char* vx_version(void) { return "voxsim-gb300 0.1 (sm_103a)"; }
const char* vx_last_error(void) { return g_err.c_str(); }

int vx_plan_counts(const vx_desc* desc, int64_t* n_voxels, int64_t* n_bonds, int64_t* n_surface) {
  Lattice L;
  int rc = build_lattice(desc, L, g_err);
  if (rc) return rc;
  if (n_voxels) *n_voxels = L.N;
  if (n_bonds) *n_bonds = L.n_bonds;
  if (n_surface) *n_surface = L.n_surface;
  return VX_OK;
}

int vx_plan_dt(const vx_desc* desc, const float* log_E, float dt_factor, double* dt_out) {
  if (!dt_out) return fail(VX_ERR_ARG, "dt_out is NULL");
  if (!(dt_factor > 0.f)) return fail(VX_ERR_ARG, "dt_factor must be positive");
  Lattice L;
  int rc = build_lattice(desc, L, g_err);
  if (rc) return rc;
  std::vector<double> dt;
  stable_dt(L, log_E, dt_factor, dt);
  std::copy(dt.begin(), dt.end(), dt_out);
  return VX_OK;
}

int vx_region_mask(const vx_desc* desc, int32_t body, const float loc[3], const float size[3], uint8_t* mask,
                   int64_t* n_out) {
  if (!loc || !size || !mask) return fail(VX_ERR_ARG, "loc, size and mask are required");
  Lattice L;
  int rc = build_lattice(desc, L, g_err);
  if (rc) return rc;
  if (body < 0 || body >= L.n_bodies) return fail(VX_ERR_ARG, "body out of range");
  int64_t n = region_mask(L, body, loc, size, mask);
  if (n_out) *n_out = n;
  return VX_OK;
}

int vx_create(const vx_desc* desc, vx_sim** out) {
  if (!out) return fail(VX_ERR_ARG, "out is NULL");
  *out = nullptr;
  vx_sim* s = new (std::nothrow) vx_sim();
  if (!s) return fail(VX_ERR_OOM, "host allocation failed");
  int rc = build_lattice(desc, s->L, g_err);
  if (rc) { delete s; return rc; }
  if (cudaGetDevice(&s->device) != cudaSuccess) { delete s; return fail(VX_ERR_CUDA, "no CUDA device"); }
  const Lattice& L = s->L;
  int64_t N = L.N;
  s->pitch = (N + 31) / 32 * 32;
  if ((rc = dalloc(&s->st, NPLANE * s->pitch)) || (rc = dalloc(&s->bf, 27 * s->pitch)) ||
      (rc = dalloc(&s->flags, N)) || (rc = dalloc(&s->mat, N)) || (rc = dalloc(&s->lat, N)) ||
      (rc = dalloc(&s->nbr, 6 * N)) || (rc = dalloc(&s->mats, L.palette.size())) ||
      (rc = dalloc(&s->dtb, L.n_bodies)) || (rc = dalloc(&s->origin, 3 * L.n_bodies)) ||
      (rc = dalloc(&s->status, 4)) || (rc = dalloc(&s->vmax, L.n_bodies)) ||
      (L.n_bodies > 1 && (rc = dalloc(&s->body, N)))) {
    vx_destroy(s);
    return rc;
  }
  auto up = [&](void* d, const void* h, size_t n) { return cudaMemcpy(d, h, n, cudaMemcpyHostToDevice); };
  if (up(s->mat, L.mat.data(), N) || up(s->lat, L.lat.data(), N * 4) || up(s->nbr, L.nbr.data(), 6 * N * 4) ||
      up(s->origin, L.origin.data(), 3 * L.n_bodies * 4) ||
      (s->body && up(s->body, L.body.data(), N * 4)) || cudaMemset(s->flags, 0, N) ||
      cudaMemset(s->status, 0, 16) || cudaMemset(s->vmax, 0, 4 * L.n_bodies) ||
      cudaMemset(s->bf, 0, sizeof(float) * 27 * s->pitch)) {
    vx_destroy(s);
    return fail(VX_ERR_CUDA, "upload failed");
  }
  quant_params(L.l, &s->qK, &s->qQ);
  if ((rc = upload_materials(s)) || (rc = recompute_dt(s)) || (rc = vx_reset(s, nullptr))) {
    vx_destroy(s);
    return rc;
  }
  *out = s;
  return VX_OK;
}

void vx_destroy(vx_sim* s) {
  if (!s) return;
  cudaSetDevice(s->device);
  dfree(s->st); dfree(s->bf); dfree(s->flags); dfree(s->mat); dfree(s->lat); dfree(s->body); dfree(s->nbr);
  dfree(s->phase); dfree(s->logE); dfree(s->fext); dfree(s->mats); dfree(s->dtb); dfree(s->origin);
  dfree(s->status); dfree(s->stage); dfree(s->surf); dfree(s->sidx); dfree(s->xq); dfree(s->bucket);
  dfree(s->hcount); dfree(s->hcursor); dfree(s->hstart); dfree(s->bsum); dfree(s->sorted); dfree(s->ccount);
  dfree(s->cand); dfree(s->acc); dfree(s->vmax); dfree(s->cflag); dfree(s->any); dfree(s->nreb);
  delete s;
}

int vx_get_counts(vx_sim* s, int64_t* n_voxels, int64_t* n_bonds, int64_t* n_surface) {
  if (!s) return fail(VX_ERR_ARG, "sim is NULL");
  if (n_voxels) *n_voxels = s->L.N;
  if (n_bonds) *n_bonds = s->L.n_bonds;
  if (n_surface) *n_surface = s->L.n_surface;
  return VX_OK;
}

int vx_get_anchors(vx_sim* s, double* anchors) {
  if (!s || !anchors) return fail(VX_ERR_ARG, "sim and anchors are required");
  const Lattice& L = s->L;
  double l = L.l;
  for (int64_t v = 0; v < L.N; ++v) {
    int b = L.body[v];
    uint32_t p = L.lat[v];
    int c[3] = {lat_i(p), lat_j(p), lat_k(p)};
    for (int a = 0; a < 3; ++a) anchors[3 * v + a] = (double)L.origin[3 * b + a] + (c[a] + 0.5) * l;
  }
  return VX_OK;
}

int vx_set_materials(vx_sim* s, const vx_material* palette, int32_t n) {
  int rc = check_sim(s);
  if (rc) return rc;
  if (!palette || n != (int32_t)s->L.palette.size()) return fail(VX_ERR_ARG, "palette size must match the lattice's");
  for (int m = 0; m < n; ++m) {
    const vx_material& p = palette[m];
    if (!(p.E > 0.f) || !(p.rho > 0.f) || !(p.nu > -1.f && p.nu < 0.5f) || !(p.mu_s >= 0.f) || !(p.mu_k >= 0.f))
      return fail(VX_ERR_ARG, "material out of range");
  }
  s->L.palette.assign(palette, palette + n);
  if ((rc = upload_materials(s)) || (rc = recompute_dt(s))) return rc;
  update_threshold(s);
  return VX_OK;
}

int vx_set_voxel_params(vx_sim* s, const float* log_E, const float* phase) {
  int rc = check_sim(s);
  if (rc) return rc;
  int64_t N = s->L.N;
  if (log_E) {
    for (int64_t v = 0; v < N; ++v)
      if (!std::isfinite(log_E[v])) return fail(VX_ERR_ARG, "log_E must be finite");
    if (!s->logE && (rc = dalloc(&s->logE, N))) return rc;
    s->logE_h.assign(log_E, log_E + N);
    VX_CUDA(cudaMemcpy(s->logE, log_E, N * 4, cudaMemcpyHostToDevice));
    if ((rc = recompute_dt(s))) return rc;
  }
  if (phase) {
    if (!s->phase && (rc = dalloc(&s->phase, N))) return rc;
    VX_CUDA(cudaMemcpy(s->phase, phase, N * 4, cudaMemcpyHostToDevice));
    s->has_phase = true;
  }
  return VX_OK;
}

int vx_set_fixed_mask(vx_sim* s, const uint8_t* mask) {
  int rc = check_sim(s);
  if (rc) return rc;
  if (!mask) return fail(VX_ERR_ARG, "mask is NULL");
  int64_t N = s->L.N;
  std::vector<uint8_t> f(N);
  VX_CUDA(cudaMemcpy(f.data(), s->flags, N, cudaMemcpyDeviceToHost));
  for (int64_t v = 0; v < N; ++v) f[v] = (uint8_t)((f[v] & ~1u) | (mask[v] ? 1u : 0u));
  VX_CUDA(cudaMemcpy(s->flags, f.data(), N, cudaMemcpyHostToDevice));
  return VX_OK;
}

int vx_add_fixed_region(vx_sim* s, int32_t body, const float loc[3], const float size[3], int64_t* n_out) {
  int rc = check_sim(s);
  if (rc) return rc;
  if (!loc || !size || body < 0 || body >= s->L.n_bodies) return fail(VX_ERR_ARG, "bad region");
  int64_t N = s->L.N;
  std::vector<uint8_t> m(N), f(N);
  int64_t n = region_mask(s->L, body, loc, size, m.data());
  VX_CUDA(cudaMemcpy(f.data(), s->flags, N, cudaMemcpyDeviceToHost));
  for (int64_t v = 0; v < N; ++v) if (m[v]) f[v] |= 1u;
  VX_CUDA(cudaMemcpy(s->flags, f.data(), N, cudaMemcpyHostToDevice));
  // fixed voxels are immobile: zero their velocities
  std::vector<float> st(NPLANE * (size_t)s->pitch);
  VX_CUDA(cudaMemcpy(st.data(), s->st, st.size() * 4, cudaMemcpyDeviceToHost));
  for (int64_t v = 0; v < N; ++v)
    if (m[v]) for (int p = VX; p <= WZ; ++p) st[(size_t)p * s->pitch + v] = 0.f;
  VX_CUDA(cudaMemcpy(s->st, st.data(), st.size() * 4, cudaMemcpyHostToDevice));
  if (n_out) *n_out = n;
  return VX_OK;
}

int vx_add_forced_region(vx_sim* s, int32_t body, const float loc[3], const float size[3], const float F[3],
                         int64_t* n_out) {
  int rc = check_sim(s);
  if (rc) return rc;
  if (!loc || !size || !F || body < 0 || body >= s->L.n_bodies) return fail(VX_ERR_ARG, "bad region");
  int64_t N = s->L.N;
  std::vector<uint8_t> m(N);
  int64_t n = region_mask(s->L, body, loc, size, m.data());
  if (n_out) *n_out = n;
  if (n == 0) return VX_OK;
  if (!s->fext) {
    if ((rc = dalloc(&s->fext, 3 * s->pitch))) return rc;
    VX_CUDA(cudaMemset(s->fext, 0, 12 * s->pitch));
  }
  std::vector<float> f(3 * (size_t)s->pitch);
  VX_CUDA(cudaMemcpy(f.data(), s->fext, f.size() * 4, cudaMemcpyDeviceToHost));
  for (int64_t v = 0; v < N; ++v)
    if (m[v]) for (int a = 0; a < 3; ++a) f[(size_t)a * s->pitch + v] += (float)((double)F[a] / (double)n);
  VX_CUDA(cudaMemcpy(s->fext, f.data(), f.size() * 4, cudaMemcpyHostToDevice));
  s->has_fext = true;
  return VX_OK;
}

int vx_set_forces(vx_sim* s, const float* F) {
  int rc = check_sim(s);
  if (rc) return rc;
  if (!F) { s->has_fext = false; return VX_OK; }
  int64_t N = s->L.N;
  if (!s->fext && (rc = dalloc(&s->fext, 3 * s->pitch))) return rc;
  std::vector<float> f(3 * (size_t)s->pitch, 0.f);
  for (int64_t v = 0; v < N; ++v) for (int a = 0; a < 3; ++a) f[(size_t)a * s->pitch + v] = F[3 * v + a];
  VX_CUDA(cudaMemcpy(s->fext, f.data(), f.size() * 4, cudaMemcpyHostToDevice));
  s->has_fext = true;
  return VX_OK;
}

int vx_set_damping(vx_sim* s, float zb, float zg, float zc) {
  if (!s) return fail(VX_ERR_ARG, "sim is NULL");
  if (!(zb >= 0.f) || !(zg >= 0.f) || !(zc >= 0.f)) return fail(VX_ERR_ARG, "damping ratios must be >= 0");
  s->zb = zb; s->zg = zg; s->zc = zc;
  return VX_OK;
}

int vx_set_environment(vx_sim* s, float gravity_z, int32_t floor_on, int32_t collide_on) {
  int rc = check_sim(s);
  if (rc) return rc;
  if (!std::isfinite(gravity_z)) return fail(VX_ERR_ARG, "gravity must be finite");
  s->gz = gravity_z;
  s->floor_on = floor_on ? 1 : 0;
  int was = s->collide_on;
  s->collide_on = collide_on ? 1 : 0;
  if (s->collide_on && !was) {
    if ((rc = force_rebuild(s, 0))) return rc;
    VX_CUDA(cudaDeviceSynchronize());
  }
  return VX_OK;
}

int vx_set_actuation(vx_sim* s, float amplitude, int64_t period, float offset) {
  if (!s) return fail(VX_ERR_ARG, "sim is NULL");
  if (period < 0 || !std::isfinite(amplitude) || !std::isfinite(offset)) return fail(VX_ERR_ARG, "bad actuation");
  s->actA = amplitude; s->actP = period; s->actT0 = offset;
  update_threshold(s);
  return VX_OK;
}

int vx_set_dt_factor(vx_sim* s, float f) {
  int rc = check_sim(s);
  if (rc) return rc;
  if (!(f > 0.f && f <= 1.f)) return fail(VX_ERR_ARG, "dt_factor must be in (0, 1]");
  s->dt_factor = f;
  return recompute_dt(s);
}

int vx_get_dt(vx_sim* s, double* dt) {
  if (!s || !dt) return fail(VX_ERR_ARG, "sim and dt are required");
  std::copy(s->dt.begin(), s->dt.end(), dt);
  return VX_OK;
}

int vx_set_dt(vx_sim* s, const double* dt) {
  int rc = check_sim(s);
  if (rc) return rc;
  if (!dt) return fail(VX_ERR_ARG, "dt is NULL");
  for (int b = 0; b < s->L.n_bodies; ++b)
    if (!(dt[b] > 0.0) || !std::isfinite(dt[b])) return fail(VX_ERR_ARG, "dt must be positive");
  s->dt.assign(dt, dt + s->L.n_bodies);
  return upload_dt(s);
}

int vx_reset(vx_sim* s, const float v0[3]) {
  int rc = check_sim(s);
  if (rc) return rc;
  launch_reset_state(s->st, s->pitch, (int)s->L.N, s->flags, v0 ? v0[0] : 0.f, v0 ? v0[1] : 0.f,
                     v0 ? v0[2] : 0.f, 0);
  VX_CUDA(cudaGetLastError());
  VX_CUDA(cudaMemset(s->status, 0, 16));
  VX_CUDA(cudaMemset(s->vmax, 0, 4 * s->L.n_bodies));
  s->step = 0;
  if (s->collide_on && (rc = force_rebuild(s, 0))) return rc;
  VX_CUDA(cudaDeviceSynchronize());
  return VX_OK;
}

int vx_read_state(vx_sim* s, const vx_state_view* out, int32_t dst_on_device, void* stream) {
  int rc = check_sim(s);
  if (rc) return rc;
  if (!out) return fail(VX_ERR_ARG, "view is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  int N = (int)s->L.N;
  if (dst_on_device) {
    launch_pack_state(s->st, s->pitch, N, s->flags, out->offset, out->quat, out->vel, out->angvel, out->flags, st);
    VX_CUDA(cudaGetLastError());
    VX_CUDA(cudaStreamSynchronize(st));
    return VX_OK;
  }
  if ((rc = ensure_stage(s))) return rc;
  float* off = s->stage;
  float* quat = off + 3 * (size_t)N;
  float* vel = quat + 4 * (size_t)N;
  float* w = vel + 3 * (size_t)N;
  uint8_t* fl = (uint8_t*)(w + 3 * (size_t)N);
  launch_pack_state(s->st, s->pitch, N, s->flags, out->offset ? off : nullptr, out->quat ? quat : nullptr,
                    out->vel ? vel : nullptr, out->angvel ? w : nullptr, out->flags ? fl : nullptr, st);
  VX_CUDA(cudaGetLastError());
  if (out->offset) VX_CUDA(cudaMemcpyAsync(out->offset, off, 12 * (size_t)N, cudaMemcpyDeviceToHost, st));
  if (out->quat) VX_CUDA(cudaMemcpyAsync(out->quat, quat, 16 * (size_t)N, cudaMemcpyDeviceToHost, st));
  if (out->vel) VX_CUDA(cudaMemcpyAsync(out->vel, vel, 12 * (size_t)N, cudaMemcpyDeviceToHost, st));
  if (out->angvel) VX_CUDA(cudaMemcpyAsync(out->angvel, w, 12 * (size_t)N, cudaMemcpyDeviceToHost, st));
  if (out->flags) VX_CUDA(cudaMemcpyAsync(out->flags, fl, (size_t)N, cudaMemcpyDeviceToHost, st));
  VX_CUDA(cudaStreamSynchronize(st));
  return VX_OK;
}

int vx_write_state(vx_sim* s, const vx_state_view* in, int32_t src_on_device, void* stream) {
  int rc = check_sim(s);
  if (rc) return rc;
  if (!in) return fail(VX_ERR_ARG, "view is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  int N = (int)s->L.N;
  if (src_on_device) {
    launch_unpack_state(s->st, s->pitch, N, s->flags, in->offset, in->quat, in->vel, in->angvel, in->flags, st);
    VX_CUDA(cudaGetLastError());
    VX_CUDA(cudaStreamSynchronize(st));
    return VX_OK;
  }
  if ((rc = ensure_stage(s))) return rc;
  float* off = s->stage;
  float* quat = off + 3 * (size_t)N;
  float* vel = quat + 4 * (size_t)N;
  float* w = vel + 3 * (size_t)N;
  uint8_t* fl = (uint8_t*)(w + 3 * (size_t)N);
  if (in->offset) VX_CUDA(cudaMemcpyAsync(off, in->offset, 12 * (size_t)N, cudaMemcpyHostToDevice, st));
  if (in->quat) VX_CUDA(cudaMemcpyAsync(quat, in->quat, 16 * (size_t)N, cudaMemcpyHostToDevice, st));
  if (in->vel) VX_CUDA(cudaMemcpyAsync(vel, in->vel, 12 * (size_t)N, cudaMemcpyHostToDevice, st));
  if (in->angvel) VX_CUDA(cudaMemcpyAsync(w, in->angvel, 12 * (size_t)N, cudaMemcpyHostToDevice, st));
  if (in->flags) VX_CUDA(cudaMemcpyAsync(fl, in->flags, (size_t)N, cudaMemcpyHostToDevice, st));
  launch_unpack_state(s->st, s->pitch, N, s->flags, in->offset ? off : nullptr, in->quat ? quat : nullptr,
                      in->vel ? vel : nullptr, in->angvel ? w : nullptr, in->flags ? fl : nullptr, st);
  VX_CUDA(cudaGetLastError());
  VX_CUDA(cudaStreamSynchronize(st));
  return VX_OK;
}

int vx_get_step(vx_sim* s, int64_t* step) {
  if (!s || !step) return fail(VX_ERR_ARG, "sim and step are required");
  *step = s->step;
  return VX_OK;
}

int vx_set_step(vx_sim* s, int64_t step) {
  if (!s || step < 0) return fail(VX_ERR_ARG, "bad step");
  s->step = step;
  return VX_OK;
}

int vx_step_async(vx_sim* s, int64_t n, void* stream) {
  int rc = check_sim(s);
  if (rc) return rc;
  if (n < 0) return fail(VX_ERR_ARG, "n_steps must be >= 0");
  cudaStream_t st = (cudaStream_t)stream;
  StepArgs A = step_args(s);
  CollideArgs C;
  if (s->collide_on) C = collide_args(s);
  for (int64_t i = 0; i < n; ++i) {
    A.step = s->step + i;
    launch_step(A, st);
    if (s->collide_on) {
      launch_horizon(C, st);
      launch_rebuild(C, st);
    }
  }
  s->step += n;
  VX_CUDA(cudaGetLastError());
  return VX_OK;
}

int vx_get_status(vx_sim* s, void* stream, int32_t* status, int64_t* bad_step, int64_t* bad_voxel) {
  int rc = check_sim(s);
  if (rc) return rc;
  int h[4] = {0, -1, 0, 0};
  VX_CUDA(cudaMemcpyAsync(h, s->status, 16, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
  VX_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  int code = VX_OK;
  if (h[0] & kStatusUnstable) code = VX_ERR_UNSTABLE;
  else if (h[0] & kStatusCapacity) code = VX_ERR_CAPACITY;
  long long bs;
  std::memcpy(&bs, &h[2], 8);
  if (status) *status = code;
  if (bad_step) *bad_step = (h[0] & kStatusUnstable) ? bs : -1;
  if (bad_voxel) *bad_voxel = (h[0] & kStatusUnstable) ? h[1] : -1;
  return VX_OK;
}

int vx_step(vx_sim* s, int64_t n, void* stream) {
  int rc = vx_step_async(s, n, stream);
  if (rc) return rc;
  int32_t code;
  int64_t bs, bv;
  if ((rc = vx_get_status(s, stream, &code, &bs, &bv))) return rc;
  if (code == VX_ERR_UNSTABLE)
    return fail(code, "non-finite state at step " + std::to_string(bs) + ", voxel " + std::to_string(bv));
  if (code == VX_ERR_CAPACITY)
    return fail(code, "collision candidate list overflow (more than " + std::to_string(kCandCap) + " per voxel)");
  return VX_OK;
}

int vx_rebuild_collisions(vx_sim* s, void* stream) {
  int rc = check_sim(s);
  if (rc) return rc;
  if ((rc = force_rebuild(s, (cudaStream_t)stream))) return rc;
  VX_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  return VX_OK;
}

int vx_get_collision_pairs(vx_sim* s, int32_t* pairs, int64_t cap, int64_t* n_out) {
  int rc = check_sim(s);
  if (rc) return rc;
  if (cap > 0 && !pairs) return fail(VX_ERR_ARG, "pairs is NULL");
  int64_t S = s->L.n_surface;
  if (!s->coll_alloc || S == 0) { if (n_out) *n_out = 0; return VX_OK; }
  VX_CUDA(cudaDeviceSynchronize());
  std::vector<int32_t> cnt(S), cand(S * kCandCap);
  VX_CUDA(cudaMemcpy(cnt.data(), s->ccount, S * 4, cudaMemcpyDeviceToHost));
  VX_CUDA(cudaMemcpy(cand.data(), s->cand, S * kCandCap * 4, cudaMemcpyDeviceToHost));
  int64_t n = 0;
  for (int64_t i = 0; i < S; ++i) {
    int32_t v = s->L.surf_list[i];
    for (int c = 0; c < cnt[i]; ++c) {
      int32_t j = cand[i * kCandCap + c];
      if (j <= v) continue;
      if (n < cap) { pairs[2 * n] = v; pairs[2 * n + 1] = j; }
      ++n;
    }
  }
  if (n_out) *n_out = n;
  return VX_OK;
}

int vx_collision_stats(vx_sim* s, int64_t* n_rebuilds, double* accumulator) {
  int rc = check_sim(s);
  if (rc) return rc;
  long long nr = 0;
  float a = 0.f;
  if (s->coll_alloc) {
    VX_CUDA(cudaDeviceSynchronize());
    VX_CUDA(cudaMemcpy(&nr, s->nreb, 8, cudaMemcpyDeviceToHost));
    VX_CUDA(cudaMemcpy(&a, s->acc, 4, cudaMemcpyDeviceToHost));
  }
  if (n_rebuilds) *n_rebuilds = nr;
  if (accumulator) *accumulator = a;
  return VX_OK;
}

}  // extern "C"

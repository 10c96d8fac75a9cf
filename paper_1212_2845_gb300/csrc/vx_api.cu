// C ABI of the simulator (declared in include/vx.h): argument checking,
// device memory ownership and the launch sequence of each step.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <tuple>
#include <string>
#include <vector>

#include "vx.h"
#include "vx_host.h"
#include "vx_kernels.h"

using namespace vx;

namespace {

// Named range on the profiler timeline (NVTX; free when no tool is attached).
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};

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

// Fault injection for tests: VX_DEVICE_ALLOC_CAP=<bytes> in the environment
// makes every larger device allocation fail as out of memory.
bool over_alloc_cap(size_t bytes) {
  const char* c = std::getenv("VX_DEVICE_ALLOC_CAP");
  if (!c || !*c) return false;
  char* end = nullptr;
  const unsigned long long cap = std::strtoull(c, &end, 10);
  return end && *end == 0 && bytes > cap;
}

template <class T> int dalloc(T** p, size_t n) {
  *p = nullptr;
  if (n == 0) n = 1;
  if (over_alloc_cap(n * sizeof(T)))
    return fail(VX_ERR_OOM, "device allocation of " + std::to_string(n * sizeof(T)) +
                                " bytes is above VX_DEVICE_ALLOC_CAP");
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

int vx::set_error(int code, const std::string& msg) { return fail(code, msg); }

int vx::status_code(int bits) {
  if (bits & kStatusUnstable) return VX_ERR_UNSTABLE;
  if (bits & kStatusTimeout) return VX_ERR_TIMEOUT;
  if (bits & kStatusCapacity) return VX_ERR_CAPACITY;
  if (bits & kStatusArg) return VX_ERR_ARG;
  if (bits & kStatusBounds) return VX_ERR_BOUNDS;
  return VX_OK;
}

struct vx_sim {
  Lattice L;
  Tiling T;
  int device = 0;
  int64_t pitch = 0;
  int form = VX_FORM_PIPELINED;
  int tile_max = 256;
  size_t smem = 0;
  int cur = 0;             // index of the buffer holding the current state
  // parameters
  float zb = 1.f, zg = 0.f, zc = 1.f, gz = 0.f;
  int floor_on = 0, collide_on = 0;
  float actA = 0.f, actT0 = 0.f;
  int64_t actP = 0;
  float actC = 0.f;       // fl(2 pi / actP): the actuation angle's step
  // per-material temperature signals (amplitude, offset, phase shift); an
  // empty vector means the global value (phase shift 0)
  std::vector<float> mactA, mactT0, mactPh;
  bool act_any = false;    // some material has a non-zero temperature offset
  float dt_factor = 0.9f;
  float v0[3] = {0.f, 0.f, 0.f};  // initial velocity of a reset without one
  std::vector<double> dt;
  std::vector<float> logE_h;
  std::vector<float> fext_h;   // canonical order, 3 per voxel
  std::vector<int32_t> surf_h; // surface voxels, internal order
  int64_t step = 0;
  bool has_phase = false, has_fext = false;
  // device buffers (internal order)
  float* st = nullptr;     // two state buffers of NPLANE * pitch floats
  float* bf = nullptr;     // two-pass bond results (allocated on first use)
  int32_t* iperm = nullptr;
  int32_t* perm = nullptr;  // internal -> canonical (state writes)
  int4* tile_a = nullptr;
  int4* tile_b = nullptr;
  int32_t* halo = nullptr;
  uint16_t* plus = nullptr;
  uint32_t* hbonds = nullptr;
  int32_t* tdesc = nullptr;   // pipelined form
  int32_t* hfix = nullptr;
  uint32_t* vw = nullptr;
  uint2* plus2 = nullptr;
  size_t pipe_smem = 0;
  int pipe_grid = 0;
  // multi-step form (one cooperative launch for n steps)
  int multistep = 1;          // 1: multi-step launches for vx_step(n > 1) (resident form on small
                              // lattices, else the cooperative grid launch); 2: grid launch only
  int multi_grid = 0;
  int multi_co = 0;           // co-resident CTAs of the multi-step kernel
  unsigned* bar = nullptr;    // grid barrier words
  int64_t bar_spins = 1ll << 24;  // barrier wait budget in 128-cycle units: about one second
  int32_t bar_extra = 0;      // phantom CTAs (fault injection)
  // batched form
  int64_t group_voxels = 0;   // 0: off; VX_GROUPS_RESIDENT: the shared-memory-resident form
  // resident form: groups of whole bodies kept in the shared memory of a CTA
  // cluster for all steps of a launch (planned per model configuration)
  int res_ok = -1;            // -1 not planned for res_cfg, 0 not possible, 1 planned
  uint64_t res_cfg = ~0ull;
  int res_C = 0, res_cap = 0, res_grid = 0, res_threads = 0;
  bool res_per_voxel = false;  // bond phase split: thread per voxel (many groups) or per bond (one wave)
  size_t res_smem = 0;
  int32_t* r_grp = nullptr;
  int32_t* r_cls = nullptr;
  int32_t* r_clg = nullptr;
  Batch B;
  int32_t* b_cta_start = nullptr;
  int32_t* b_cta_groups = nullptr;
  int32_t* b_group_tiles = nullptr;
  size_t batch_smem = 0;
  uint8_t* mask = nullptr;
  uint8_t* flags = nullptr;
  uint8_t* mat = nullptr;
  uint32_t* lat = nullptr;
  int32_t* body = nullptr;
  int32_t* nbr = nullptr;
  float* phase = nullptr;
  float* logE = nullptr;
  float* fext = nullptr;
  DevMat* mats = nullptr;
  float* lut = nullptr;    // material-pair bond constants (n_mats <= kLutMaxMats)
  float* dtb = nullptr;
  float* origin = nullptr;
  int* status = nullptr;
  float* stage = nullptr;
  // collisions
  bool coll_alloc = false;
  int coll_all = 0;          // candidates among all voxels (not only surface voxels)
  int coll_every = 0;        // rebuild every step (not on the horizon trigger)
  int64_t coll_S = 0;        // voxels in the candidate search
  int H = 0, qK = 0;
  int64_t qQ = 0;
  float threshold = 0.f;
  int32_t* surf = nullptr;
  int32_t* sidx = nullptr;
  int64_t* xq = nullptr;
  int4* cell = nullptr;
  uint32_t* bucket = nullptr;
  uint32_t* hcount = nullptr;
  uint32_t* hcursor = nullptr;
  uint32_t* hstart = nullptr;
  uint32_t* bsum = nullptr;
  int32_t* sorted = nullptr;
  int4* scell = nullptr;     // searched voxels in bucket order: cell and index
  int64_t* sxq = nullptr;    // quantised coordinates (3 planes)
  int4* sinf = nullptr;      // voxel, lattice word, body
  int32_t* ccount = nullptr;
  int32_t* vcnt = nullptr;   // per voxel: candidate count (staged by the step)
  unsigned* dmax = nullptr;  // per body: largest displacement of a state write (float bits)
  int32_t* cand = nullptr;
  float* acc = nullptr;
  unsigned* vmax = nullptr;
  int* cflag = nullptr;
  int* any = nullptr;
  unsigned* hdone = nullptr;  // CTAs of a step launch done (the step keeps the horizon)
  long long* nreb = nullptr;
  unsigned* cbar = nullptr;  // grid barrier words of the rebuild launch
  int64_t* qorg = nullptr;   // shared world: quantised body origins rint(origin 2^K), 3 per body
  // adjoint form
  uint64_t gen = 0;           // bumped by every call that changes the state or the model
  uint64_t cfg = 0;           // bumped by every call that changes the model or the step form
  // captured batched launch (vx_graph_capture)
  cudaGraphExec_t gexec = nullptr;
  int64_t g_n = 0;            // steps per replay
  uint64_t g_cfg = 0;         // cfg at capture
  int64_t* ctr_d = nullptr;   // device (step, buffer) read by the captured kernel
  int64_t ctr_h[2] = {0, 0};
  // FP64 audit
  double* aud = nullptr;      // per-body origins, per-material values, block partials, result
  unsigned* vmax_d = nullptr; // relaxation: largest speed (float bits)
  uint64_t ro_gen = 0;        // gen at the end of the recorded rollout
  int64_t ro_steps = 0;       // steps of the recorded rollout (0: none)
  int ro_K = 0;               // checkpoint interval
  int64_t ro_step0 = 0;       // step counter at the rollout start
  int64_t ro_cap = 0;         // checkpoints allocated
  float* ro_ckpt = nullptr;   // ro_cap x NPLANE x pitch floats
  uint8_t* ro_cfl = nullptr;  // ro_cap x pitch flag bytes
  int ro_seg_cap = 0;         // states of the segment buffer
  float* ro_seg = nullptr;    // ro_seg_cap x NPLANE x pitch floats
  uint8_t* ro_sfl = nullptr;  // ro_seg_cap x pitch flag bytes
  float* ro_sfm = nullptr;    // (ro_seg_cap - 1) x 6 x pitch floats: bond sums of every segment step
  size_t adj_smem = 0;        // dynamic shared memory adj_tile is prepared for
  float* adj = nullptr;       // adjoint work planes (adjoint_args)
  float* cw = nullptr;        // per voxel m_v / (mass of its body)
  int32_t* bstart = nullptr;  // internal index range of every body (n_bodies + 1)
  float* loss_d = nullptr;    // per body loss
  float* wb_d = nullptr;      // per body loss weight
};

namespace {

float* cur_state(vx_sim* s) { return s->st + (size_t)s->cur * NPLANE * s->pitch; }
float* next_state(vx_sim* s) { return s->st + (size_t)(1 - s->cur) * NPLANE * s->pitch; }

StepArgs step_args(vx_sim* s) {
  StepArgs A;
  A.h_done = nullptr;  // the horizon is kept by a separate launch unless the caller sets it
  A.h_acc = nullptr;
  A.h_flag = A.h_any = nullptr;
  A.h_threshold = 0.f;
  A.h_world = 0;
  A.n_bodies = s->L.n_bodies;
  A.N = (int)s->L.N;
  A.pitch = s->pitch;
  A.l = s->L.l;
  A.st_in = cur_state(s);
  A.st_out = next_state(s);
  A.flags = s->flags;
  A.mat = s->mat;
  A.lat = s->lat;
  A.body = s->body;
  A.nbr = s->nbr;
  A.phase = s->has_phase ? s->phase : nullptr;
  A.logE = s->logE_h.empty() ? nullptr : s->logE;
  A.fext = s->has_fext ? s->fext : nullptr;
  A.mats = s->mats;
  A.n_mats = (int)s->L.palette.size();
  A.lut = (s->lut && s->logE_h.empty()) ? s->lut : nullptr;
  A.dt_body = s->dtb;
  A.origin = s->origin;
  A.bf = s->bf;
  A.zb = s->zb; A.zg = s->zg; A.zc = s->zc; A.gz = s->gz;
  A.floor_on = s->floor_on;
  A.collide_on = s->collide_on;
  A.actA = s->actA; A.actT0 = s->actT0;
  A.act_on = s->act_any ? 1 : 0;
  A.act_w = 0.f;
  A.step = s->step;
  A.tile_a = s->tile_a;
  A.tile_b = s->tile_b;
  A.halo = s->halo;
  A.plus = s->plus;
  A.hbonds = s->hbonds;
  A.tdesc = s->tdesc;
  A.hfix = s->hfix;
  A.hstride = s->T.halo_stride;
  A.vw = s->vw;
  A.plus2 = s->plus2;
  A.mask = s->mask;
  A.n_tiles = (int)s->T.n_tiles();
  A.max_local = s->T.max_local;
  A.sidx = s->sidx;
  A.ccount = s->ccount;
  A.vcnt = s->vcnt;
  A.cand = s->cand;
  A.vmax_bits = s->vmax;
  A.status = s->status;
  A.fm_out = nullptr;
  return A;
}

CollideArgs collide_args(vx_sim* s) {
  CollideArgs C;
  C.S = (int)s->coll_S;
  C.n_bodies = s->L.n_bodies;
  C.H = s->H;
  C.K = s->qK;
  C.Q = s->qQ;
  C.ostride_v = 4;           // offsets are the x, y, z of state plane A
  C.ostride_a = 1;
  C.threshold = s->threshold;
  C.st = cur_state(s);
  C.surf = s->surf;
  C.lat = s->lat;
  C.body = s->body;
  C.dt_body = s->dtb;
  C.xq = s->xq;
  C.cell = s->cell;
  C.bucket = s->bucket;
  C.hcount = s->hcount;
  C.hcursor = s->hcursor;
  C.hstart = s->hstart;
  C.bsum = s->bsum;
  C.sorted = s->sorted;
  C.scell = s->scell;
  C.sxq = s->sxq;
  C.sinf = s->sinf;
  C.ccount = s->ccount;
  C.vcnt = s->vcnt;
  C.cand = s->cand;
  C.acc = s->acc;
  C.vmax_bits = s->vmax;
  C.flag = s->cflag;
  C.any = s->any;
  C.n_rebuilds = s->nreb;
  C.status = s->status;
  C.bar = s->cbar;
  C.spins = s->bar_spins;
  C.extra = (unsigned)s->bar_extra;
  C.qorg = s->collide_on == 2 ? s->qorg : nullptr;
  return C;
}

// Temperature signal of material i (Sec 2.3): its own amplitude, offset and
// phase shift where set, else the global ones; no period, no oscillation.
void material_signal(const vx_sim* s, size_t i, float* a, float* t0, float* ph) {
  *a = s->mactA.empty() ? s->actA : s->mactA[i];
  *t0 = s->mactT0.empty() ? s->actT0 : s->mactT0[i];
  *ph = s->mactPh.empty() ? 0.f : s->mactPh[i];
  if (s->actP == 0) *a = 0.f;
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
    float a, t0, ph;
    material_signal(s, i, &a, &t0, &ph);
    m[i].act_A = a; m[i].act_T0 = t0; m[i].act_phase = ph;
  }
  s->act_any = false;
  for (const DevMat& d : m) s->act_any = s->act_any || d.act_A != 0.f || d.act_T0 != 0.f;
  VX_CUDA(cudaMemcpy(s->mats, m.data(), m.size() * sizeof(DevMat), cudaMemcpyHostToDevice));
  return VX_OK;
}

constexpr int kLutMaxMats = 16;

// Bond constants of every material pair (Sec 2.1.1, 2.1.2, 2.1.5) in double,
// used when no per-voxel stiffness is set: a1, a2, b2, b3, c/2, c/4, cr/2.
int upload_lut(vx_sim* s) {
  int nm = (int)s->L.palette.size();
  if (nm > kLutMaxMats) return VX_OK;
  if (!s->lut) {
    int rc = dalloc(&s->lut, (size_t)8 * nm * nm);
    if (rc) return rc;
  }
  std::vector<float> h((size_t)8 * nm * nm, 0.f);
  const double l = s->L.l;
  for (int i = 0; i < nm; ++i)
    for (int j = 0; j < nm; ++j) {
      const vx_material& p = s->L.palette[i];
      const vx_material& q = s->L.palette[j];
      double E1 = p.E, E2 = q.E;
      double G1 = E1 / (2.0 * (1.0 + (double)p.nu)), G2 = E2 / (2.0 * (1.0 + (double)q.nu));
      double Ec = 2.0 * E1 * E2 / (E1 + E2), Gc = 2.0 * G1 * G2 / (G1 + G2);
      double m1 = (double)p.rho * l * l * l, m2 = (double)q.rho * l * l * l;
      double mmin = std::min(m1, m2), Imin = mmin * l * l / 6.0;
      double a1 = Ec * l, a2 = Gc * l * l * l / 6.0, b2 = Ec * l * l / 2.0, b3 = Ec * l * l * l / 6.0;
      float* e = &h[(size_t)8 * (i * nm + j)];
      e[0] = (float)a1; e[1] = (float)a2; e[2] = (float)b2; e[3] = (float)b3;
      double c = 2.0 * s->zb * std::sqrt(mmin * a1), cr = 2.0 * s->zb * std::sqrt(Imin * b3);
      e[4] = (float)(c / 2.0);
      e[5] = (float)(c / 4.0);
      e[6] = (float)(cr / 2.0);
    }
  VX_CUDA(cudaMemcpy(s->lut, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice));
  return VX_OK;
}

int upload_dt(vx_sim* s) {
  std::vector<float> f(s->dt.size());
  for (size_t b = 0; b < f.size(); ++b) f[b] = (float)s->dt[b];
  VX_CUDA(cudaMemcpy(s->dtb, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice));
  return VX_OK;
}

int ensure_nbr(vx_sim* s);
std::vector<int64_t> body_ranges(const vx_sim* s);

// Largest w^2 of every body's bonds and contact springs, reduced in FP32 on
// the device from the uploaded lattice (materials, per-voxel moduli, bonds).
// The neighbour planes are uploaded for the call when no step form holds them.
int device_w2(vx_sim* s, std::vector<float>& w2) {
  const Lattice& L = s->L;
  const int nb = L.n_bodies;
  const bool had_nbr = s->nbr != nullptr;
  int rc = ensure_nbr(s);
  if (rc) return rc;
  const std::vector<int64_t> bs = body_ranges(s);
  std::vector<int4> ch;
  for (int b = 0; b < nb; ++b)
    for (int64_t v = bs[b]; v < bs[b + 1]; v += kDtChunk)
      ch.push_back(make_int4((int)v, (int)std::min<int64_t>(v + kDtChunk, bs[b + 1]), b, 0));
  std::vector<unsigned> bits(nb, 0u);
  int4* ch_d = nullptr;
  unsigned* w2_d = nullptr;
  rc = dalloc(&ch_d, std::max<size_t>(ch.size(), 1));
  if (!rc) rc = dalloc(&w2_d, nb);
  if (!rc) {
    cudaError_t e = cudaMemcpy(ch_d, ch.data(), ch.size() * sizeof(int4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(w2_d, 0, nb * sizeof(unsigned));
    if (e == cudaSuccess) {
      DtArgs D;
      D.n_chunks = (int)ch.size();
      D.N = L.N;
      D.l = L.l;
      D.mat = s->mat;
      D.logE = s->logE_h.empty() ? nullptr : s->logE;
      D.nbr = s->nbr;
      D.mats = s->mats;
      D.chunks = ch_d;
      D.w2 = w2_d;
      launch_stable_w2(D, 0);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(bits.data(), w2_d, nb * sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) rc = fail(VX_ERR_CUDA, std::string("stable timestep reduction: ") + cudaGetErrorString(e));
  }
  dfree(ch_d);
  dfree(w2_d);
  if (!had_nbr) dfree(s->nbr);
  w2.resize(nb);
  for (int b = 0; b < nb; ++b) std::memcpy(&w2[b], &bits[b], sizeof(float));
  return rc;
}

// dt = f / (2 pi w_max) per body (Sec 2.1.4) from the device reduction's
// largest w^2 (FP32); the host forms the square root and the quotient in
// FP64, and the step uses dt rounded to FP32.
int recompute_dt(vx_sim* s) {
  std::vector<float> w2;
  int rc = device_w2(s, w2);
  if (rc) return rc;
  s->dt.assign(s->L.n_bodies, 0.0);
  for (int b = 0; b < s->L.n_bodies; ++b)
    s->dt[b] = w2[b] > 0.f ? (double)s->dt_factor / (2.0 * M_PI * std::sqrt((double)w2[b])) : 0.0;
  if (s->collide_on == 2) {  // one world, one clock: every body takes the smallest timestep
    double dmin = 0.0;
    for (double d : s->dt)
      if (d > 0.0 && (dmin == 0.0 || d < dmin)) dmin = d;
    for (double& d : s->dt) d = dmin;
  }
  return upload_dt(s);
}

void update_threshold(vx_sim* s) {
  double smax = 0.0;  // largest thermal strain any material can reach
  for (size_t i = 0; i < s->L.palette.size(); ++i) {
    float a, t0, ph;
    material_signal(s, i, &a, &t0, &ph);
    smax = std::max(smax, std::fabs((double)s->L.palette[i].cte) *
                              (std::fabs((double)t0) + std::fabs((double)a)));
  }
  double l = s->L.l;
  double cmax = l * (1.0 + smax);
  s->threshold = (float)(2.0 * l - cmax);
}

int alloc_collisions(vx_sim* s) {
  if (s->coll_alloc) return VX_OK;
  const Lattice& L = s->L;
  int64_t S = s->coll_all ? L.N : L.n_surface;
  s->coll_S = S;
  int H = 1024;
  while ((int64_t)H < 2 * S) H <<= 1;
  s->H = H;
  int rc;
  if ((rc = dalloc(&s->surf, S)) || (rc = dalloc(&s->sidx, L.N)) || (rc = dalloc(&s->xq, 3 * S)) ||
      (rc = dalloc(&s->cell, S)) ||
      (rc = dalloc(&s->bucket, S)) || (rc = dalloc(&s->hcount, H)) || (rc = dalloc(&s->hcursor, H)) ||
      (rc = dalloc(&s->hstart, H + 1)) || (rc = dalloc(&s->bsum, kRebuildMaxGrid)) || (rc = dalloc(&s->cbar, 2)) ||
      (rc = dalloc(&s->sorted, S)) || (rc = dalloc(&s->scell, S)) || (rc = dalloc(&s->sxq, 3 * S)) ||
      (rc = dalloc(&s->sinf, S)) || (rc = dalloc(&s->ccount, S)) || (rc = dalloc(&s->cand, S * kCandCap)) ||
      (rc = dalloc(&s->vcnt, L.N)) || (rc = dalloc(&s->dmax, L.n_bodies)) ||
      (rc = dalloc(&s->acc, L.n_bodies)) || (rc = dalloc(&s->cflag, L.n_bodies)) || (rc = dalloc(&s->any, 1)) ||
      (rc = dalloc(&s->hdone, 1)) ||
      (rc = dalloc(&s->nreb, 1)))
    return rc;
  // searched voxels (surface voxels, or all) in ascending internal order
  std::vector<int32_t> surf(S), sidx(L.N, -1);
  for (int64_t i = 0; i < S; ++i) surf[i] = s->coll_all ? (int32_t)i : s->T.iperm[L.surf_list[i]];
  std::sort(surf.begin(), surf.end());
  for (int64_t i = 0; i < S; ++i) sidx[surf[i]] = (int32_t)i;
  s->surf_h = surf;
  VX_CUDA(cudaMemcpy(s->surf, surf.data(), S * sizeof(int32_t), cudaMemcpyHostToDevice));
  VX_CUDA(cudaMemcpy(s->sidx, sidx.data(), L.N * sizeof(int32_t), cudaMemcpyHostToDevice));
  VX_CUDA(cudaMemset(s->ccount, 0, std::max<int64_t>(S, 1) * sizeof(int32_t)));
  VX_CUDA(cudaMemset(s->vcnt, 0, L.N * sizeof(int32_t)));
  VX_CUDA(cudaMemset(s->dmax, 0, L.n_bodies * sizeof(unsigned)));
  VX_CUDA(cudaMemset(s->acc, 0, L.n_bodies * sizeof(float)));
  VX_CUDA(cudaMemset(s->cflag, 0, L.n_bodies * sizeof(int)));
  VX_CUDA(cudaMemset(s->any, 0, sizeof(int)));
  VX_CUDA(cudaMemset(s->hdone, 0, sizeof(unsigned)));
  VX_CUDA(cudaMemset(s->nreb, 0, sizeof(long long)));
  VX_CUDA(cudaMemset(s->cbar, 0, 2 * sizeof(unsigned)));
  s->coll_alloc = true;
  return VX_OK;
}

void free_collisions(vx_sim* s) {
  dfree(s->surf); dfree(s->sidx); dfree(s->xq); dfree(s->cell); dfree(s->bucket); dfree(s->hcount); dfree(s->hcursor);
  dfree(s->hstart); dfree(s->bsum); dfree(s->cbar); dfree(s->sorted); dfree(s->ccount); dfree(s->cand);
  dfree(s->scell); dfree(s->sxq); dfree(s->sinf); dfree(s->vcnt); dfree(s->dmax);
  dfree(s->acc); dfree(s->cflag); dfree(s->any); dfree(s->nreb); dfree(s->hdone);
  s->coll_alloc = false;
  s->coll_S = 0;
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
  return dalloc(&s->stage, (size_t)14 * s->L.N);  // 13 floats + the flag bytes
}

// canonical-order host array -> internal-order device array
template <class T> int upload_permuted(vx_sim* s, T* dst, const T* src, int planes, int64_t plane_stride) {
  int64_t N = s->L.N;
  std::vector<T> h((size_t)planes * plane_stride, T(0));
  for (int p = 0; p < planes; ++p)
    for (int64_t c = 0; c < N; ++c) h[(size_t)p * plane_stride + s->T.iperm[c]] = src[(size_t)planes * c + p];
  VX_CUDA(cudaMemcpy(dst, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
  return VX_OK;
}

int upload_tiling(vx_sim* s) {
  const Tiling& T = s->T;
  int64_t nt = T.n_tiles();
  dfree(s->tile_a); dfree(s->tile_b); dfree(s->halo); dfree(s->plus); dfree(s->hbonds);
  dfree(s->tdesc); dfree(s->hfix); dfree(s->vw); dfree(s->plus2);
  int rc;
  const int64_t N = s->L.N;
  if ((rc = dalloc(&s->tile_a, nt)) || (rc = dalloc(&s->tile_b, nt)) || (rc = dalloc(&s->halo, T.halo.size())) ||
      (rc = dalloc(&s->plus, T.plus.size())) || (rc = dalloc(&s->hbonds, T.halo_bonds.size())) ||
      (rc = dalloc(&s->tdesc, T.tile_desc.size())) || (rc = dalloc(&s->hfix, T.halo_fixed.size())) ||
      (rc = dalloc(&s->vw, N)) || (rc = dalloc(&s->plus2, N)))
    return rc;
  {
    std::vector<uint32_t> vw(N);
    std::vector<uint2> p2(N);
    for (int64_t v = 0; v < N; ++v) {
      vw[v] = (uint32_t)s->L.mat[T.perm[v]] | (uint32_t)T.mask[v] << 8;
      p2[v].x = (uint32_t)T.plus[v] | (uint32_t)T.plus[(size_t)N + v] << 16;
      p2[v].y = (uint32_t)T.plus[2 * (size_t)N + v] | 0xFFFF0000u;
    }
    VX_CUDA(cudaMemcpy(s->vw, vw.data(), N * 4, cudaMemcpyHostToDevice));
    VX_CUDA(cudaMemcpy(s->plus2, p2.data(), N * 8, cudaMemcpyHostToDevice));
    VX_CUDA(cudaMemcpy(s->tdesc, T.tile_desc.data(), T.tile_desc.size() * 4, cudaMemcpyHostToDevice));
    VX_CUDA(cudaMemcpy(s->hfix, T.halo_fixed.data(), T.halo_fixed.size() * 4, cudaMemcpyHostToDevice));
  }
  VX_CUDA(cudaMemcpy(s->tile_a, T.tile_a.data(), nt * sizeof(int4), cudaMemcpyHostToDevice));
  VX_CUDA(cudaMemcpy(s->tile_b, T.tile_b.data(), nt * sizeof(int4), cudaMemcpyHostToDevice));
  if (!T.halo.empty()) VX_CUDA(cudaMemcpy(s->halo, T.halo.data(), T.halo.size() * 4, cudaMemcpyHostToDevice));
  VX_CUDA(cudaMemcpy(s->plus, T.plus.data(), T.plus.size() * 2, cudaMemcpyHostToDevice));
  if (!T.halo_bonds.empty())
    VX_CUDA(cudaMemcpy(s->hbonds, T.halo_bonds.data(), T.halo_bonds.size() * 4, cudaMemcpyHostToDevice));
  int nm = (int)s->L.palette.size();
  s->smem = fused_smem_bytes(s->tile_max, nm, nm <= kLutMaxMats);
  if (prepare_fused(s->tile_max, s->smem) != 0)
    return fail(VX_ERR_CUDA, "fused kernel needs " + std::to_string(s->smem) + " bytes of shared memory");
  return VX_OK;
}

// Shared memory of the pipelined kernels for the optional arrays in use;
// (re)prepares the persistent kernel when it changes.
int ensure_pipe(vx_sim* s, const StepArgs& A) {
  int nm = (int)s->L.palette.size();
  size_t sm = pipe_smem_bytes(s->tile_max, A.phase != nullptr, A.logE != nullptr, A.body != nullptr,
                              A.fext != nullptr, A.collide_on != 0, nm, nm <= kLutMaxMats);
  if (sm != s->pipe_smem) {
    if (prepare_pipe(s->tile_max, sm, &s->pipe_grid) != 0 || prepare_batched(s->tile_max, sm) != 0 ||
        prepare_multi(s->tile_max, sm, (int)s->T.n_tiles(), &s->multi_grid, &s->multi_co) != 0)
      return fail(VX_ERR_CUDA, "pipelined kernels need " + std::to_string(sm) + " bytes of shared memory");
    s->pipe_smem = sm;
  }
  return VX_OK;
}

// Bodies' internal voxel ranges, n_bodies + 1 offsets (bodies are contiguous
// in the internal order).
std::vector<int64_t> body_ranges(const vx_sim* s) {
  const Lattice& L = s->L;
  std::vector<int64_t> bs(L.n_bodies + 1, L.N);
  int prev = -1;
  for (int64_t v = 0; v < L.N; ++v) {
    const int b = L.body[s->T.perm[v]];
    for (int k = prev + 1; k <= b; ++k) bs[k] = v;
    prev = b;
  }
  return bs;
}

int ensure_nbr(vx_sim* s) {
  if (s->nbr) return VX_OK;
  const int64_t N = s->L.N;
  int rc;
  if ((rc = dalloc(&s->nbr, 6 * N))) return rc;
  std::vector<int32_t> nb(6 * (size_t)N);
  for (int sl = 0; sl < 6; ++sl)
    for (int64_t c = 0; c < N; ++c) {
      int32_t u = s->L.nbr[(size_t)sl * N + c];
      nb[(size_t)sl * N + s->T.iperm[c]] = u < 0 ? -1 : s->T.iperm[u];
    }
  VX_CUDA(cudaMemcpy(s->nbr, nb.data(), nb.size() * 4, cudaMemcpyHostToDevice));
  return VX_OK;
}

// lattices up to this size step n > 1 in the resident form by default (one
// cluster of up to 8 CTAs holds them)
constexpr int64_t kResidentAutoVoxels = 8192;

bool is_resident(int64_t g) {
  return g == VX_GROUPS_RESIDENT || g == VX_GROUPS_RESIDENT_BOND || g == VX_GROUPS_RESIDENT_VOXEL;
}

// Plans the resident form for the current model.  Split: a thread per bond
// when every group gets a cluster of its own (one wave: the phases' chains
// set the time), else a thread per voxel.  Slice capacity: 1,024 voxels per
// CTA for the per-bond split (a small lattice spread over up to 8 CTAs);
// 512 for the per-voxel split where the largest body allows it, so that two
// CTAs share an SM and one computes while the other waits at its cluster
// barrier, with as many threads as half the largest slice (two voxels per
// thread).  Cluster size: the smallest power of two that holds the largest
// body (at most 16).  Sets res_ok.
int ensure_resident(vx_sim* s) {
  if (s->res_cfg == s->cfg && s->res_ok >= 0) return VX_OK;
  s->res_cfg = s->cfg;
  s->res_ok = 0;
  int rc;
  if ((rc = ensure_nbr(s))) return rc;
  const Lattice& L = s->L;
  const int nm = (int)L.palette.size();
  const bool fext = s->has_fext, lut = s->lut && s->logE_h.empty();
  int dev = 0, optin = 0, n_sm = 0;
  VX_CUDA(cudaGetDevice(&dev));
  VX_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  VX_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
  const std::vector<int64_t> bs = body_ranges(s);
  int64_t max_body = 0;
  for (int b = 0; b < L.n_bodies; ++b) max_body = std::max(max_body, bs[b + 1] - bs[b]);
  auto cluster_for = [&](int cap) { int C = 1; while ((int64_t)C * cap < max_body) C *= 2; return C; };
  int cap = 1024;
  while (cap > 64 && res_smem_bytes(cap, fext, nm, lut) > (size_t)optin) cap -= 32;
  if (res_smem_bytes(cap, fext, nm, lut) > (size_t)optin) return VX_OK;
  int C = cluster_for(cap);
  if (C > 16) return VX_OK;
  ResPlan P;
  plan_resident(bs, (int64_t)C * cap, 1, P);
  const int64_t ng1 = (int64_t)P.grp_start.size() - 1;
  bool per_voxel;
  if (s->group_voxels == VX_GROUPS_RESIDENT_VOXEL) per_voxel = true;
  else if (s->group_voxels == VX_GROUPS_RESIDENT_BOND) per_voxel = false;
  else per_voxel = ng1 * C > n_sm;  // more groups than one wave of clusters
  int threads = kResThreads;
  if (per_voxel) {
    if (cluster_for(512) <= 16) { cap = 512; C = cluster_for(cap); }
    plan_resident(bs, (int64_t)C * cap, 1, P);
    int64_t max_slice = 0;
    for (size_t g = 0; g + 1 < P.grp_start.size(); ++g)
      max_slice = std::max<int64_t>(max_slice, (P.grp_start[g + 1] - P.grp_start[g] + C - 1) / C);
    threads = (int)std::min<int64_t>(kResThreads, std::max<int64_t>(32, ((max_slice + 1) / 2 + 31) / 32 * 32));
  } else {
    while (C < 8 && ng1 * C * 2 <= n_sm) C *= 2;  // spread a small lattice over more SMs
    plan_resident(bs, (int64_t)C * cap, 1, P);
  }
  const size_t smem = res_smem_bytes(cap, fext, nm, lut);
  int max_cl = 0;
  for (;;) {
    max_cl = 0;
    if (prepare_resident(C, threads, smem, fext, per_voxel, &max_cl) == 0 || C == 1 ||
        (int64_t)(C / 2) * cap < max_body)
      break;
    C /= 2;
  }
  if (max_cl < 1) return VX_OK;
  plan_resident(bs, (int64_t)C * cap, 1, P);
  const int ng = (int)P.grp_start.size() - 1;
  const int n_cl = std::min(ng, max_cl);
  plan_resident(bs, (int64_t)C * cap, n_cl, P);
  dfree(s->r_grp); dfree(s->r_cls); dfree(s->r_clg);
  if ((rc = dalloc(&s->r_grp, P.grp_start.size())) || (rc = dalloc(&s->r_cls, P.cl_start.size())) ||
      (rc = dalloc(&s->r_clg, P.cl_groups.size())))
    return rc;
  VX_CUDA(cudaMemcpy(s->r_grp, P.grp_start.data(), P.grp_start.size() * 4, cudaMemcpyHostToDevice));
  VX_CUDA(cudaMemcpy(s->r_cls, P.cl_start.data(), P.cl_start.size() * 4, cudaMemcpyHostToDevice));
  VX_CUDA(cudaMemcpy(s->r_clg, P.cl_groups.data(), P.cl_groups.size() * 4, cudaMemcpyHostToDevice));
  s->res_C = C;
  s->res_cap = cap;
  s->res_threads = threads;
  s->res_grid = n_cl * C;
  s->res_smem = smem;
  s->res_per_voxel = per_voxel;
  s->res_ok = 1;
  return VX_OK;
}

ResArgs res_args(vx_sim* s, int64_t n) {
  ResArgs R;
  R.grp_start = s->r_grp;
  R.cl_start = s->r_cls;
  R.cl_groups = s->r_clg;
  R.buf0 = s->st;
  R.buf1 = s->st + (size_t)NPLANE * s->pitch;
  R.cur0 = s->cur;
  R.n_steps = (int)n;
  R.step0 = s->step;
  R.act_P = s->actP;
  R.act_c = s->actC;
  R.ctr = nullptr;
  R.cap = s->res_cap;
  return R;
}

int ensure_two_pass(vx_sim* s) {
  int rc;
  if ((rc = ensure_nbr(s))) return rc;
  if (s->bf) return VX_OK;
  if ((rc = dalloc(&s->bf, 27 * s->pitch))) return rc;
  VX_CUDA(cudaMemset(s->bf, 0, sizeof(float) * 27 * s->pitch));
  return VX_OK;
}

// Group schedule of the batched form for the current tiling and grid.
int build_schedule(vx_sim* s) {
  std::vector<int64_t> starts = batch_group_starts(s->L, s->group_voxels);
  build_batch(s->T, starts, s->L.N, s->pipe_grid, s->B);
  dfree(s->b_cta_start); dfree(s->b_cta_groups); dfree(s->b_group_tiles);
  int rc;
  if ((rc = dalloc(&s->b_cta_start, s->B.cta_start.size())) ||
      (rc = dalloc(&s->b_cta_groups, std::max<size_t>(1, s->B.cta_groups.size()))) ||
      (rc = dalloc(&s->b_group_tiles, s->B.group_tiles.size())))
    return rc;
  VX_CUDA(cudaMemcpy(s->b_cta_start, s->B.cta_start.data(), s->B.cta_start.size() * 4, cudaMemcpyHostToDevice));
  if (!s->B.cta_groups.empty())
    VX_CUDA(cudaMemcpy(s->b_cta_groups, s->B.cta_groups.data(), s->B.cta_groups.size() * 4, cudaMemcpyHostToDevice));
  VX_CUDA(cudaMemcpy(s->b_group_tiles, s->B.group_tiles.data(), s->B.group_tiles.size() * 4, cudaMemcpyHostToDevice));
  return VX_OK;
}

// Rebuild the tiles for the current tile size (with group boundaries when
// the batched form is on) and upload them.
//
// Without batching the persistent grid (G CTAs) walks the tiles round robin,
// so on a lattice of a few tiles per CTA the step lasts as long as the CTAs
// that walk one tile more than the others.  There the runs are shortened to
// about N / (k G) voxels (k = tiles per CTA at full length) so that every
// CTA walks k tiles; never below half the tile size, and only while k <= 8
// (beyond that the last round is a small part of the step).
int retile(vx_sim* s, int tile_max) {
  Tiling T;
  std::vector<int64_t> starts;
  if (s->group_voxels > 0) starts = batch_group_starts(s->L, s->group_voxels);
  int run = tile_max;
  int64_t G = 0, k = 0;
  int dev = 0, n_sm = 0;
  if (s->group_voxels == 0 && cudaGetDevice(&dev) == cudaSuccess &&
      cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n_sm > 0) {
    G = (int64_t)n_sm * (tile_max == 128 ? 4 : (tile_max == 256 ? 2 : 1));  // resident CTAs of the pipelined kernels
    k = (s->L.N + (int64_t)tile_max * G - 1) / ((int64_t)tile_max * G);
    const int64_t r = (s->L.N + k * G - 1) / (k * G);
    if (k <= 8 && 2 * r >= tile_max && r < tile_max) run = (int)r;
  }
  int rc;
  for (int pass = 0;; ++pass) {
    rc = build_tiling(s->L, run, 2 * tile_max, T, g_err, s->group_voxels > 0 ? &starts : nullptr);
    if (rc) return rc;
    // tiles shortened around large halos can leave a few more than k G:
    // shorten the runs in proportion (at most two more passes)
    if (run == tile_max || T.n_tiles() <= k * G || pass == 2) break;
    const int r = (int)((int64_t)run * k * G / T.n_tiles());
    if (2 * r < tile_max || r >= run) break;
    run = r;
  }
  s->T.tile_a.swap(T.tile_a); s->T.tile_b.swap(T.tile_b); s->T.halo.swap(T.halo); s->T.plus.swap(T.plus);
  s->T.halo_bonds.swap(T.halo_bonds); s->T.tile_desc.swap(T.tile_desc); s->T.halo_fixed.swap(T.halo_fixed);
  s->T.halo_stride = T.halo_stride;
  s->T.tile_max = tile_max;
  s->T.max_local = T.max_local;
  s->tile_max = tile_max;
  s->pipe_smem = 0;  // re-prepare the pipelined kernels
  s->B = Batch();
  return upload_tiling(s);
}

// read-modify-write of the flag bytes in canonical order
int edit_flags(vx_sim* s, const std::function<void(int64_t c, uint8_t& f)>& fn) {
  int64_t N = s->L.N;
  std::vector<uint8_t> f(N);
  VX_CUDA(cudaMemcpy(f.data(), s->flags, N, cudaMemcpyDeviceToHost));
  for (int64_t c = 0; c < N; ++c) fn(c, f[s->T.iperm[c]]);
  VX_CUDA(cudaMemcpy(s->flags, f.data(), N, cudaMemcpyHostToDevice));
  return VX_OK;
}


BatchArgs batch_args(vx_sim* s, int64_t n) {
  BatchArgs Bt;
  Bt.cta_start = s->b_cta_start;
  Bt.cta_groups = s->b_cta_groups;
  Bt.group_tiles = s->b_group_tiles;
  Bt.buf0 = s->st;
  Bt.buf1 = s->st + (size_t)NPLANE * s->pitch;
  Bt.cur0 = s->cur;
  Bt.n_steps = (int)n;
  Bt.step0 = s->step;
  Bt.act_P = s->actP;
  Bt.act_c = s->actC;
  Bt.ctr = nullptr;
  return Bt;
}

// ---- adjoint form ----------------------------------------------------------
float act_phase(const vx_sim* s, int64_t step) { return act_angle(step, s->actP, s->actC); }

// One step from A.st_in to A.st_out with the simulator's per-step form.
int launch_form_step(vx_sim* s, const StepArgs& A, cudaStream_t st) {
  if (s->form == VX_FORM_PIPELINED) {
    int rc = ensure_pipe(s, A);
    if (rc) return rc;
    launch_pipe(A, s->tile_max, s->pipe_smem, s->pipe_grid, st);
  } else {
    launch_step(A, s->form, s->tile_max, s->smem, st);
  }
  return VX_OK;
}

// Mass weights m_v / M_body (internal order) and the bodies' internal index
// ranges for the centre-of-mass loss.
int upload_com_weights(vx_sim* s) {
  const Lattice& L = s->L;
  const int64_t N = L.N;
  const int nb = L.n_bodies;
  int rc;
  if (!s->cw && ((rc = dalloc(&s->cw, N)) || (rc = dalloc(&s->bstart, nb + 1)) || (rc = dalloc(&s->loss_d, nb)) ||
                 (rc = dalloc(&s->wb_d, nb))))
    return rc;
  const double l3 = (double)L.l * (double)L.l * (double)L.l;
  std::vector<double> M(nb, 0.0);
  for (int64_t c = 0; c < N; ++c) M[L.body[c]] += (double)L.palette[L.mat[c]].rho * l3;
  std::vector<float> cw(N);
  std::vector<int32_t> bs(nb + 1, (int32_t)N);
  int prev = -1;
  for (int64_t v = 0; v < N; ++v) {
    const int32_t c = s->T.perm[v];
    const int b = L.body[c];
    if (b < prev) return fail(VX_ERR_STATE, "bodies are not contiguous in the internal order");
    for (int k = prev + 1; k <= b; ++k) bs[k] = (int32_t)v;
    prev = b;
    cw[v] = (float)((double)L.palette[L.mat[c]].rho * l3 / M[b]);
  }
  VX_CUDA(cudaMemcpy(s->cw, cw.data(), 4 * N, cudaMemcpyHostToDevice));
  VX_CUDA(cudaMemcpy(s->bstart, bs.data(), 4 * (nb + 1), cudaMemcpyHostToDevice));
  return VX_OK;
}


// ---- batched-form autotuning ------------------------------------------------
// Size class of a lattice for the tuning cache: log2 of the voxel count, log2
// of the mean body size, and the optional per-voxel arrays that change the
// kernels' staging.
struct TuneKey {
  int lg_n, lg_body, lut, le, ph, fx;
  bool operator<(const TuneKey& o) const {
    return std::tie(lg_n, lg_body, lut, le, ph, fx) < std::tie(o.lg_n, o.lg_body, o.lut, o.le, o.ph, o.fx);
  }
};
struct TuneVal { int tile_max; int64_t group_voxels; double rate; };
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune;

int ilog2(int64_t x) { int r = 0; while (x > 1) { x >>= 1; ++r; } return r; }

TuneKey tune_key(const vx_sim* s) {
  const int64_t N = s->L.N;
  return TuneKey{ilog2(N), ilog2(std::max<int64_t>(1, N / s->L.n_bodies)),
                 (int)(s->L.palette.size() <= (size_t)kLutMaxMats && s->logE_h.empty()), (int)!s->logE_h.empty(),
                 (int)s->has_phase, (int)s->has_fext};
}

}  // namespace

extern "C" {

const char* vx_version(void) { return "voxsim-gb300 0.2 (sm_103a)"; }
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

int vx_plan_tiles(const vx_desc* desc, int32_t tile_max, int64_t* n_tiles, int64_t* n_halo, int64_t* n_tile_bonds,
                  int32_t* max_local, int32_t* max_halo_bonds) {
  Lattice L;
  int rc = build_lattice(desc, L, g_err);
  if (rc) return rc;
  Tiling T;
  if (tile_max != 128 && tile_max != 256 && tile_max != 512) return fail(VX_ERR_ARG, "tile_max must be 128, 256 or 512");
  if ((rc = build_tiling(L, tile_max, 2 * tile_max, T, g_err))) return rc;
  if (n_tiles) *n_tiles = T.n_tiles();
  if (n_halo) *n_halo = (int64_t)T.halo.size();
  if (n_tile_bonds) *n_tile_bonds = T.n_tile_bonds();
  if (max_local) *max_local = T.max_local;
  if (max_halo_bonds) *max_halo_bonds = T.max_halo_bonds;
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
  const Range range("vx_create");
  if (!out) return fail(VX_ERR_ARG, "out is NULL");
  *out = nullptr;
  vx_sim* s = new (std::nothrow) vx_sim();
  if (!s) return fail(VX_ERR_OOM, "host allocation failed");
  int rc = build_lattice(desc, s->L, g_err);
  if (!rc) rc = build_tiling(s->L, s->tile_max, 2 * s->tile_max, s->T, g_err);
  if (rc) { delete s; return rc; }
  if (cudaGetDevice(&s->device) != cudaSuccess) { delete s; return fail(VX_ERR_CUDA, "no CUDA device"); }
  const Lattice& L = s->L;
  int64_t N = L.N;
  s->pitch = (N + 31) / 32 * 32;
  if ((rc = dalloc(&s->st, 2 * NPLANE * s->pitch)) || (rc = dalloc(&s->flags, N)) || (rc = dalloc(&s->mat, N)) ||
      (rc = dalloc(&s->lat, N)) || (rc = dalloc(&s->iperm, N)) || (rc = dalloc(&s->perm, N)) || (rc = dalloc(&s->mask, N)) ||
      (rc = dalloc(&s->mats, L.palette.size())) || (rc = dalloc(&s->dtb, L.n_bodies)) ||
      (rc = dalloc(&s->origin, 3 * L.n_bodies)) || (rc = dalloc(&s->status, 8)) ||
      (rc = dalloc(&s->vmax, L.n_bodies)) || (L.n_bodies > 1 && (rc = dalloc(&s->body, N)))) {
    vx_destroy(s);
    return rc;
  }
  std::vector<uint8_t> mat(N);
  std::vector<uint32_t> lat(N);
  std::vector<int32_t> body(N);
  for (int64_t v = 0; v < N; ++v) {
    int32_t c = s->T.perm[v];
    mat[v] = L.mat[c]; lat[v] = L.lat[c]; body[v] = L.body[c];
  }
  auto up = [&](void* d, const void* h, size_t n) { return cudaMemcpy(d, h, n, cudaMemcpyHostToDevice); };
  if (up(s->mat, mat.data(), N) || up(s->lat, lat.data(), N * 4) || up(s->iperm, s->T.iperm.data(), N * 4) ||
      up(s->perm, s->T.perm.data(), N * 4) ||
      up(s->mask, s->T.mask.data(), N) || up(s->origin, L.origin.data(), 3 * L.n_bodies * 4) ||
      (s->body && up(s->body, body.data(), N * 4)) || cudaMemset(s->flags, 0, N) ||
      cudaMemset(s->status, 0, 32) || cudaMemset(s->vmax, 0, 4 * L.n_bodies) ||
      cudaMemset(s->st, 0, sizeof(float) * 2 * NPLANE * s->pitch)) {
    vx_destroy(s);
    return fail(VX_ERR_CUDA, "upload failed");
  }
  quant_params(L.l, &s->qK, &s->qQ);
  if ((rc = upload_tiling(s)) || (rc = upload_materials(s)) || (rc = upload_lut(s)) || (rc = recompute_dt(s)) ||
      (rc = vx_reset(s, nullptr))) {
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
  dfree(s->iperm); dfree(s->perm); dfree(s->tile_a); dfree(s->tile_b); dfree(s->halo); dfree(s->plus); dfree(s->hbonds); dfree(s->mask);
  dfree(s->tdesc); dfree(s->hfix); dfree(s->vw); dfree(s->plus2);
  dfree(s->phase); dfree(s->logE); dfree(s->fext); dfree(s->mats); dfree(s->lut); dfree(s->dtb); dfree(s->origin);
  dfree(s->status); dfree(s->stage); dfree(s->surf); dfree(s->sidx); dfree(s->xq); dfree(s->cell); dfree(s->bucket);
  dfree(s->hcount); dfree(s->hcursor); dfree(s->hstart); dfree(s->bsum); dfree(s->sorted); dfree(s->ccount);
  dfree(s->cand); dfree(s->acc); dfree(s->vmax); dfree(s->cflag); dfree(s->any); dfree(s->nreb); dfree(s->hdone);
  dfree(s->scell); dfree(s->sxq); dfree(s->sinf); dfree(s->vcnt); dfree(s->dmax);
  dfree(s->ro_ckpt); dfree(s->ro_cfl); dfree(s->ro_seg); dfree(s->ro_sfl); dfree(s->ro_sfm); dfree(s->adj);
  dfree(s->cw);
  dfree(s->bstart); dfree(s->loss_d); dfree(s->wb_d); dfree(s->ctr_d); dfree(s->aud); dfree(s->bar); dfree(s->vmax_d); dfree(s->cbar); dfree(s->qorg);
  dfree(s->r_grp); dfree(s->r_cls); dfree(s->r_clg);
  if (s->gexec) cudaGraphExecDestroy(s->gexec);
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

int vx_set_step_form(vx_sim* s, int32_t form, int32_t tile_max) {
  if (s) ++s->cfg;  // invalidates a captured graph
  int rc = check_sim(s);
  if (rc) return rc;
  if (form != VX_FORM_FUSED && form != VX_FORM_TWO_PASS && form != VX_FORM_PIPELINED)
    return fail(VX_ERR_ARG, "unknown step form");
  if (form == VX_FORM_TWO_PASS && (rc = ensure_two_pass(s))) return rc;
  if (form != VX_FORM_TWO_PASS && tile_max != 0 && tile_max != s->tile_max) {
    if (tile_max != 128 && tile_max != 256 && tile_max != 512) return fail(VX_ERR_ARG, "tile_max must be 128, 256 or 512");
    // the voxel order depends only on the lattice, so the state stays valid
    if ((rc = retile(s, tile_max))) return rc;
  }
  s->form = form;
  return VX_OK;
}

int vx_set_batching(vx_sim* s, int64_t group_voxels) {
  if (s) ++s->cfg;  // invalidates a captured graph
  int rc = check_sim(s);
  if (rc) return rc;
  if (is_resident(group_voxels)) {
    if (s->form == VX_FORM_TWO_PASS) return fail(VX_ERR_STATE, "the resident form needs a fused form");
    const int64_t prev = s->group_voxels;
    s->group_voxels = group_voxels;  // the plan reads the requested split
    s->res_ok = -1;
    if ((rc = ensure_resident(s))) { s->group_voxels = prev; return rc; }
    if (s->res_ok != 1) {
      s->group_voxels = prev;
      return fail(VX_ERR_STATE, "the resident form does not fit this lattice (a body above 16 CTAs' shared memory)");
    }
    return retile(s, s->tile_max);
  }
  if (group_voxels < 0) return fail(VX_ERR_ARG, "group_voxels must be >= 0 or one of VX_GROUPS_RESIDENT*");
  if (group_voxels > 0 && s->form == VX_FORM_TWO_PASS) return fail(VX_ERR_STATE, "batching needs a fused form");
  if (s->tile_max == 512 && group_voxels > 0) return fail(VX_ERR_ARG, "batching takes tiles of 128 or 256 voxels");
  s->group_voxels = group_voxels;
  return retile(s, s->tile_max);
}

int vx_get_tiling(vx_sim* s, int32_t* tile_max, int64_t* n_tiles, int32_t* max_local, int64_t* smem_bytes) {
  if (!s) return fail(VX_ERR_ARG, "sim is NULL");
  if (tile_max) *tile_max = s->tile_max;
  if (n_tiles) *n_tiles = s->T.n_tiles();
  if (max_local) *max_local = s->T.max_local;
  if (smem_bytes) *smem_bytes = (int64_t)s->smem;
  return VX_OK;
}

int vx_set_materials(vx_sim* s, const vx_material* palette, int32_t n) {
  if (s) { ++s->gen; ++s->cfg; }  // invalidates a recorded rollout and a captured graph
  int rc = check_sim(s);
  if (rc) return rc;
  if (!palette || n != (int32_t)s->L.palette.size()) return fail(VX_ERR_ARG, "palette size must match the lattice's");
  for (int m = 0; m < n; ++m) {
    const vx_material& p = palette[m];
    if (!(p.E > 0.f) || !(p.rho > 0.f) || !(p.nu > -1.f && p.nu < 0.5f) || !(p.mu_s >= 0.f) || !(p.mu_k >= 0.f))
      return fail(VX_ERR_ARG, "material out of range");
  }
  s->L.palette.assign(palette, palette + n);
  if ((rc = upload_materials(s)) || (rc = upload_lut(s)) || (rc = recompute_dt(s))) return rc;
  update_threshold(s);
  return VX_OK;
}

int vx_set_voxel_params(vx_sim* s, const float* log_E, const float* phase) {
  if (s) { ++s->gen; ++s->cfg; }  // invalidates a recorded rollout and a captured graph
  int rc = check_sim(s);
  if (rc) return rc;
  int64_t N = s->L.N;
  if (log_E) {
    for (int64_t v = 0; v < N; ++v)
      if (!std::isfinite(log_E[v])) return fail(VX_ERR_ARG, "log_E must be finite");
    if (!s->logE && (rc = dalloc(&s->logE, N))) return rc;
    s->logE_h.assign(log_E, log_E + N);
    if ((rc = upload_permuted(s, s->logE, log_E, 1, N))) return rc;
    if ((rc = recompute_dt(s))) return rc;
  }
  if (phase) {
    if (!s->phase && (rc = dalloc(&s->phase, N))) return rc;
    if ((rc = upload_permuted(s, s->phase, phase, 1, N))) return rc;
    s->has_phase = true;
  }
  return VX_OK;
}

int vx_set_fixed_mask(vx_sim* s, const uint8_t* mask) {
  if (s) { ++s->gen; ++s->cfg; }  // invalidates a recorded rollout and a captured graph
  int rc = check_sim(s);
  if (rc) return rc;
  if (!mask) return fail(VX_ERR_ARG, "mask is NULL");
  return edit_flags(s, [&](int64_t c, uint8_t& f) { f = (uint8_t)((f & ~1u) | (mask[c] ? 1u : 0u)); });
}

int vx_add_fixed_region(vx_sim* s, int32_t body, const float loc[3], const float size[3], int64_t* n_out) {
  if (s) { ++s->gen; ++s->cfg; }  // invalidates a recorded rollout and a captured graph
  int rc = check_sim(s);
  if (rc) return rc;
  if (!loc || !size || body < 0 || body >= s->L.n_bodies) return fail(VX_ERR_ARG, "bad region");
  int64_t N = s->L.N;
  std::vector<uint8_t> m(N);
  int64_t n = region_mask(s->L, body, loc, size, m.data());
  if ((rc = edit_flags(s, [&](int64_t c, uint8_t& f) { if (m[c]) f |= 1u; }))) return rc;
  // fixed voxels are immobile: zero their velocities in the current state
  std::vector<float> st(NPLANE * (size_t)s->pitch);
  float* cs = cur_state(s);
  VX_CUDA(cudaMemcpy(st.data(), cs, st.size() * 4, cudaMemcpyDeviceToHost));
  for (int64_t c = 0; c < N; ++c)
    if (m[c]) for (int p = VX; p <= WZ; ++p) st[state_index(p, s->T.iperm[c], s->pitch)] = 0.f;
  VX_CUDA(cudaMemcpy(cs, st.data(), st.size() * 4, cudaMemcpyHostToDevice));
  if (n_out) *n_out = n;
  return VX_OK;
}

int vx_add_forced_region(vx_sim* s, int32_t body, const float loc[3], const float size[3], const float F[3],
                         int64_t* n_out) {
  if (s) { ++s->gen; ++s->cfg; }  // invalidates a recorded rollout and a captured graph
  int rc = check_sim(s);
  if (rc) return rc;
  if (!loc || !size || !F || body < 0 || body >= s->L.n_bodies) return fail(VX_ERR_ARG, "bad region");
  int64_t N = s->L.N;
  std::vector<uint8_t> m(N);
  int64_t n = region_mask(s->L, body, loc, size, m.data());
  if (n_out) *n_out = n;
  if (n == 0) return VX_OK;
  if (s->fext_h.empty()) s->fext_h.assign(3 * (size_t)N, 0.f);
  for (int64_t c = 0; c < N; ++c)
    if (m[c]) for (int a = 0; a < 3; ++a) s->fext_h[3 * c + a] += (float)((double)F[a] / (double)n);
  return vx_set_forces(s, s->fext_h.data());
}

int vx_set_forces(vx_sim* s, const float* F) {
  if (s) { ++s->gen; ++s->cfg; }  // invalidates a recorded rollout and a captured graph
  int rc = check_sim(s);
  if (rc) return rc;
  if (!F) { s->has_fext = false; s->fext_h.clear(); return VX_OK; }
  int64_t N = s->L.N;
  if (F != s->fext_h.data()) s->fext_h.assign(F, F + 3 * N);
  if (!s->fext && (rc = dalloc(&s->fext, 3 * s->pitch))) return rc;
  if ((rc = upload_permuted(s, s->fext, F, 3, s->pitch))) return rc;
  s->has_fext = true;
  return VX_OK;
}

int vx_set_damping(vx_sim* s, float zb, float zg, float zc) {
  if (s) { ++s->gen; ++s->cfg; }  // invalidates a recorded rollout and a captured graph
  if (!s) return fail(VX_ERR_ARG, "sim is NULL");
  if (!(zb >= 0.f) || !(zg >= 0.f) || !(zc >= 0.f)) return fail(VX_ERR_ARG, "damping ratios must be >= 0");
  s->zb = zb; s->zg = zg; s->zc = zc;
  int rc = check_sim(s);
  if (rc) return rc;
  return upload_lut(s);
}

int vx_set_environment(vx_sim* s, float gravity_z, int32_t floor_on, int32_t collide_on) {
  if (s) { ++s->gen; ++s->cfg; }  // invalidates a recorded rollout and a captured graph
  int rc = check_sim(s);
  if (rc) return rc;
  if (!std::isfinite(gravity_z)) return fail(VX_ERR_ARG, "gravity must be finite");
  if (collide_on < 0 || collide_on > 2) return fail(VX_ERR_ARG, "collide_on must be 0, 1 or 2");
  s->gz = gravity_z;
  s->floor_on = floor_on ? 1 : 0;
  int was = s->collide_on;
  s->collide_on = collide_on;
  if (collide_on == 2 && !s->qorg) {
    const int nb = s->L.n_bodies;
    std::vector<int64_t> q(3 * (size_t)nb);
    for (int b = 0; b < nb; ++b)
      for (int a = 0; a < 3; ++a) q[3 * b + a] = (int64_t)std::nearbyint(std::ldexp((double)s->L.origin[3 * b + a], s->qK));
    if ((rc = dalloc(&s->qorg, q.size()))) return rc;
    VX_CUDA(cudaMemcpy(s->qorg, q.data(), q.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
  }
  if ((collide_on == 2) != (was == 2) && (rc = recompute_dt(s))) return rc;
  if (s->collide_on && s->collide_on != was) {
    if ((rc = force_rebuild(s, 0))) return rc;
    VX_CUDA(cudaDeviceSynchronize());
  }
  return VX_OK;
}

int vx_set_actuation(vx_sim* s, float amplitude, int64_t period, float offset) {
  if (s) { ++s->gen; ++s->cfg; }  // invalidates a recorded rollout and a captured graph
  if (!s) return fail(VX_ERR_ARG, "sim is NULL");
  if (period < 0 || !std::isfinite(amplitude) || !std::isfinite(offset)) return fail(VX_ERR_ARG, "bad actuation");
  if (period == 0) amplitude = 0.f;
  s->actA = amplitude; s->actP = period; s->actT0 = offset;
  s->actC = period > 0 ? (float)(2.0 * M_PI / (double)period) : 0.f;
  update_threshold(s);
  return upload_materials(s);
}

int vx_set_material_actuation(vx_sim* s, const float* amplitude, const float* offset, const float* phase) {
  if (s) { ++s->gen; ++s->cfg; }  // invalidates a recorded rollout and a captured graph
  int rc = check_sim(s);
  if (rc) return rc;
  const size_t nm = s->L.palette.size();
  for (size_t i = 0; i < nm; ++i)
    if ((amplitude && !std::isfinite(amplitude[i])) || (offset && !std::isfinite(offset[i])) ||
        (phase && !std::isfinite(phase[i])))
      return fail(VX_ERR_ARG, "material actuation values must be finite");
  if (amplitude) s->mactA.assign(amplitude, amplitude + nm); else s->mactA.clear();
  if (offset) s->mactT0.assign(offset, offset + nm); else s->mactT0.clear();
  if (phase) s->mactPh.assign(phase, phase + nm); else s->mactPh.clear();
  update_threshold(s);
  return upload_materials(s);
}

int vx_set_dt_factor(vx_sim* s, float f) {
  if (s) { ++s->gen; ++s->cfg; }  // invalidates a recorded rollout and a captured graph
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
  if (s) { ++s->gen; ++s->cfg; }  // invalidates a recorded rollout and a captured graph
  int rc = check_sim(s);
  if (rc) return rc;
  if (!dt) return fail(VX_ERR_ARG, "dt is NULL");
  for (int b = 0; b < s->L.n_bodies; ++b)
    if (!(dt[b] > 0.0) || !std::isfinite(dt[b])) return fail(VX_ERR_ARG, "dt must be positive");
  s->dt.assign(dt, dt + s->L.n_bodies);
  return upload_dt(s);
}

int vx_reset(vx_sim* s, const float v0[3]) {
  if (s) ++s->gen;  // invalidates a recorded rollout
  int rc = check_sim(s);
  if (rc) return rc;
  const float* v = v0 ? v0 : s->v0;
  launch_reset_state(cur_state(s), s->pitch, (int)s->L.N, s->flags, v[0], v[1], v[2], 0);
  VX_CUDA(cudaGetLastError());
  VX_CUDA(cudaMemset(s->status, 0, 32));
  VX_CUDA(cudaMemset(s->vmax, 0, 4 * s->L.n_bodies));
  if (s->cbar) VX_CUDA(cudaMemset(s->cbar, 0, 2 * sizeof(unsigned)));  // clean after a timed-out launch
  s->step = 0;
  if (s->collide_on && (rc = force_rebuild(s, 0))) return rc;
  VX_CUDA(cudaDeviceSynchronize());
  return VX_OK;
}

int vx_set_initial_velocity(vx_sim* s, const float v[3]) {
  if (s) ++s->gen;  // invalidates a recorded rollout
  int rc = check_sim(s);
  if (rc) return rc;
  if (!v || !std::isfinite(v[0]) || !std::isfinite(v[1]) || !std::isfinite(v[2]))
    return fail(VX_ERR_ARG, "initial velocity must be three finite values");
  for (int a = 0; a < 3; ++a) s->v0[a] = v[a];
  launch_set_velocity(cur_state(s), s->pitch, (int)s->L.N, s->flags, v[0], v[1], v[2], 0);
  VX_CUDA(cudaGetLastError());
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
    launch_pack_state(cur_state(s), s->pitch, N, s->iperm, s->flags, out->offset, out->quat, out->vel, out->angvel,
                      out->flags, st);
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
  launch_pack_state(cur_state(s), s->pitch, N, s->iperm, s->flags, out->offset ? off : nullptr,
                    out->quat ? quat : nullptr, out->vel ? vel : nullptr, out->angvel ? w : nullptr,
                    out->flags ? fl : nullptr, st);
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
  int rc = vx_write_state_async(s, in, src_on_device, stream);
  if (rc) return rc;
  VX_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  return VX_OK;
}

// With collisions on, a write is motion for the collision horizon: the
// unpack records each body's largest displacement, the accumulators grow by
// twice that, and only bodies that reach the threshold (every body after a
// rebuild that timed out or overflowed) are rebuilt.  A write that moves no
// voxel (velocities, flags, or the state just read) keeps the lists.
int write_collisions(vx_sim* s, cudaStream_t st) {
  const int rc = alloc_collisions(s);
  if (rc) return rc;
  update_threshold(s);
  const CollideArgs C = collide_args(s);
  launch_write_horizon(C, s->dmax, s->collide_on == 2, st);
  launch_rebuild(C, st);
  VX_CUDA(cudaGetLastError());
  return VX_OK;
}

int vx_write_state_async(vx_sim* s, const vx_state_view* in, int32_t src_on_device, void* stream) {
  if (s) ++s->gen;  // invalidates a recorded rollout
  int rc = check_sim(s);
  if (rc) return rc;
  if (!in) return fail(VX_ERR_ARG, "view is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  int N = (int)s->L.N;
  if (s->collide_on && (rc = alloc_collisions(s))) return rc;
  unsigned* dmax = s->collide_on ? s->dmax : nullptr;
  if (src_on_device) {
    launch_unpack_state(cur_state(s), s->pitch, N, s->perm, s->flags, in->offset, in->quat, in->vel, in->angvel,
                        in->flags, st, s->body, dmax);
    VX_CUDA(cudaGetLastError());
    return s->collide_on ? write_collisions(s, st) : VX_OK;
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
  launch_unpack_state(cur_state(s), s->pitch, N, s->perm, s->flags, in->offset ? off : nullptr,
                      in->quat ? quat : nullptr, in->vel ? vel : nullptr, in->angvel ? w : nullptr,
                      in->flags ? fl : nullptr, st, s->body, dmax);
  VX_CUDA(cudaGetLastError());
  return s->collide_on ? write_collisions(s, st) : VX_OK;
}

int vx_get_step(vx_sim* s, int64_t* step) {
  if (!s || !step) return fail(VX_ERR_ARG, "sim and step are required");
  *step = s->step;
  return VX_OK;
}

int vx_set_step(vx_sim* s, int64_t step) {
  if (s) ++s->gen;  // invalidates a recorded rollout
  if (!s || step < 0) return fail(VX_ERR_ARG, "bad step");
  s->step = step;
  return VX_OK;
}

int vx_step_async(vx_sim* s, int64_t n, void* stream) {
  const Range range("vx_step");
  if (s) ++s->gen;  // invalidates a recorded rollout
  int rc = check_sim(s);
  if (rc) return rc;
  if (n < 0) return fail(VX_ERR_ARG, "n_steps must be >= 0");
  if (n > INT32_MAX) return fail(VX_ERR_ARG, "n_steps too large for one call");
  cudaStream_t st = (cudaStream_t)stream;
  // a small lattice without collisions steps n > 1 in the resident form by
  // default: one cluster holds it for all n steps
  const bool res_auto = s->group_voxels == 0 && s->multistep == 1 && n > 1 && !s->collide_on &&
                        s->form != VX_FORM_TWO_PASS && s->L.N <= kResidentAutoVoxels;
  if (res_auto) {
    if ((rc = ensure_resident(s))) return rc;
  }
  if ((is_resident(s->group_voxels) || (res_auto && s->res_ok == 1)) && !s->collide_on && n > 0) {
    // resident form: all n steps in one launch, state in cluster shared memory
    if ((rc = ensure_resident(s))) return rc;
    if (s->res_ok != 1) return fail(VX_ERR_STATE, "the resident form does not fit this lattice");
    StepArgs A = step_args(s);
    ResArgs R = res_args(s, n);
    const cudaError_t e = launch_resident(A, R, s->res_grid, s->res_C, s->res_threads, s->res_smem, s->res_per_voxel, st);
    if (e != cudaSuccess) return fail(VX_ERR_CUDA, std::string("resident launch: ") + cudaGetErrorString(e));
    s->cur ^= (int)(n & 1);
    s->step += n;
    return VX_OK;
  }
  if (s->group_voxels > 0 && !s->collide_on && n > 0) {
    // batched form: all n steps in one launch
    StepArgs A = step_args(s);
    if ((rc = ensure_pipe(s, A))) return rc;
    if ((int64_t)s->B.cta_start.size() != (int64_t)s->pipe_grid + 1 && (rc = build_schedule(s))) return rc;
    BatchArgs Bt = batch_args(s, n);
    launch_batched(A, Bt, s->tile_max, s->pipe_smem, s->pipe_grid, st);
    s->cur ^= (int)(n & 1);
    s->step += n;
    VX_CUDA(cudaGetLastError());
    return VX_OK;
  }
  bool multi = s->multistep && s->form == VX_FORM_PIPELINED && n > 1;
  if (multi) {
    StepArgs A = step_args(s);
    if ((rc = ensure_pipe(s, A))) return rc;
    // for lattices of a few tiles per CTA, where launches and per-step ramp-up
    // dominate; on larger ones the per-step launches overlap and the barrier
    // costs more
    multi = s->T.n_tiles() <= 4 * (int64_t)s->pipe_grid;
  }
  if (multi) {
    // multi-step form: all n steps in one cooperative launch
    StepArgs A = step_args(s);
    if (!s->bar && (rc = dalloc(&s->bar, 2))) return rc;
    VX_CUDA(cudaMemsetAsync(s->bar, 0, 2 * sizeof(unsigned), st));
    MultiArgs M;
    M.buf0 = s->st;
    M.buf1 = s->st + (size_t)NPLANE * s->pitch;
    M.cur0 = s->cur;
    M.n_steps = (int)n;
    M.step0 = s->step;
    M.act_P = s->actP;
    M.act_c = s->actC;
    M.ctr = nullptr;
    M.bar = s->bar;
    M.spins = s->bar_spins;
    M.extra = (unsigned)s->bar_extra;
    M.collide = 0;
    M.every_step = 0;
    if (s->collide_on) {
      // horizon and rebuilds between the steps, on the launch's own grid and barrier
      M.collide = 1;
      M.every_step = s->coll_every ? 1 : 0;
      M.coll = collide_args(s);
      M.coll.bar = s->bar;
      M.coll.spins = s->bar_spins;
      A.h_acc = s->acc;
      A.h_flag = s->cflag;
      A.h_any = s->any;
      A.h_threshold = s->threshold;
      A.h_world = s->collide_on == 2 ? 1 : 0;
    }
    // with collisions, enough CTAs for one warp per searched voxel in a rebuild
    // (CTAs beyond the tiles meet at the barriers and join the rebuilds)
    int grid = s->multi_grid;
    if (M.collide) grid = std::max(grid, std::min(s->multi_co, (int)((s->coll_S + 7) / 8)));
    if (launch_multi(A, M, s->tile_max, s->pipe_smem, grid, st) == cudaSuccess) {
      s->cur ^= (int)(n & 1);
      s->step += n;
      return VX_OK;
    }
    cudaGetLastError();  // not co-resident on this device: fall back to one launch per step
  }
  // the pipelined step keeps the collision horizon itself (one launch less per step)
  const bool tail = s->collide_on && !s->coll_every && s->form == VX_FORM_PIPELINED;
  for (int64_t i = 0; i < n; ++i) {
    StepArgs A = step_args(s);
    if (s->actP > 0) A.act_w = act_phase(s, s->step);
    if (tail) {
      A.h_done = s->hdone;
      A.h_acc = s->acc;
      A.h_flag = s->cflag;
      A.h_any = s->any;
      A.h_threshold = s->threshold;
      A.h_world = s->collide_on == 2 ? 1 : 0;
    }
    if (s->form == VX_FORM_PIPELINED) {
      if ((rc = ensure_pipe(s, A))) return rc;
      launch_pipe(A, s->tile_max, s->pipe_smem, s->pipe_grid, st);
    } else {
      launch_step(A, s->form, s->tile_max, s->smem, st);
    }
    s->cur = 1 - s->cur;
    s->step += 1;
    if (s->collide_on) {
      CollideArgs C = collide_args(s);
      if (s->coll_every) launch_flag_all(C, st);  // rebuild every step
      else if (!tail) launch_horizon(C, st);
      launch_rebuild(C, st);
    }
  }
  VX_CUDA(cudaGetLastError());
  return VX_OK;
}

int vx_get_status(vx_sim* s, void* stream, int32_t* status, int64_t* bad_step, int64_t* bad_voxel) {
  int rc = check_sim(s);
  if (rc) return rc;
  int h[4] = {0, -1, 0, 0};
  VX_CUDA(cudaMemcpyAsync(h, s->status, 16, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
  VX_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  const int code = status_code(h[0]);
  long long bs;
  std::memcpy(&bs, &h[2], 8);
  if (status) *status = code;
  if (bad_step) *bad_step = (h[0] & kStatusUnstable) ? bs : -1;
  if (bad_voxel) *bad_voxel = (h[0] & kStatusUnstable) ? s->T.perm[h[1]] : -1;
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
  if (code == VX_ERR_TIMEOUT) return fail(code, "a grid barrier of the multi-step launch gave up waiting");
  if (code == VX_ERR_BOUNDS) {
    int h[8] = {0};
    VX_CUDA(cudaMemcpy(h, s->status, 32, cudaMemcpyDeviceToHost));
    return fail(code, "an index failed its bounds check at site " + std::to_string(h[4]) + " (index " +
                          std::to_string(h[5]) + ")");
  }
  return VX_OK;
}

int vx_rebuild_collisions(vx_sim* s, void* stream) {
  const Range range("vx_rebuild_collisions");
  int rc = check_sim(s);
  if (rc) return rc;
  if ((rc = force_rebuild(s, (cudaStream_t)stream))) return rc;
  int h[4] = {0, 0, 0, 0};
  VX_CUDA(cudaMemcpyAsync(h, s->status, 16, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
  VX_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  if (h[0] & kStatusTimeout) return fail(VX_ERR_TIMEOUT, "a grid barrier of the candidate rebuild gave up waiting");
  if (h[0] & kStatusCapacity)
    return fail(VX_ERR_CAPACITY, "collision candidate list overflow (more than " + std::to_string(kCandCap) + " per voxel)");
  return VX_OK;
}

int vx_get_collision_pairs(vx_sim* s, int32_t* pairs, int64_t cap, int64_t* n_out) {
  int rc = check_sim(s);
  if (rc) return rc;
  if (cap > 0 && !pairs) return fail(VX_ERR_ARG, "pairs is NULL");
  int64_t S = s->coll_S;
  if (!s->coll_alloc || S == 0) { if (n_out) *n_out = 0; return VX_OK; }
  VX_CUDA(cudaDeviceSynchronize());
  std::vector<int32_t> cnt(S), cand(S * kCandCap);
  VX_CUDA(cudaMemcpy(cnt.data(), s->ccount, S * 4, cudaMemcpyDeviceToHost));
  VX_CUDA(cudaMemcpy(cand.data(), s->cand, S * kCandCap * 4, cudaMemcpyDeviceToHost));
  std::vector<std::pair<int32_t, int32_t>> pr;
  for (int64_t i = 0; i < S; ++i) {
    int32_t a = s->T.perm[s->surf_h[i]];
    for (int c = 0; c < cnt[i]; ++c) {
      int32_t b = s->T.perm[cand[i * kCandCap + c]];
      if (a < b) pr.emplace_back(a, b);
    }
  }
  std::sort(pr.begin(), pr.end());
  int64_t n = (int64_t)pr.size();
  for (int64_t k = 0; k < n && k < cap; ++k) { pairs[2 * k] = pr[k].first; pairs[2 * k + 1] = pr[k].second; }
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

int vx_rollout_forward(vx_sim* s, int64_t n, int32_t K, float* loss_body, void* stream) {
  const Range range("vx_rollout_forward");
  int rc = check_sim(s);
  if (rc) return rc;
  if (n < 1 || K < 1) return fail(VX_ERR_ARG, "n_steps and checkpoint_every must be >= 1");
  if (s->collide_on) return fail(VX_ERR_STATE, "the adjoint form does not support voxel-voxel collisions");
  cudaStream_t st = (cudaStream_t)stream;
  s->ro_steps = 0;
  const int64_t N = s->L.N, P = s->pitch;
  const size_t sb = (size_t)NPLANE * P;
  const int64_t nck = (n + K - 1) / K;
  if (nck > s->ro_cap) {
    dfree(s->ro_ckpt);
    dfree(s->ro_cfl);
    s->ro_cap = 0;
    if ((rc = dalloc(&s->ro_ckpt, nck * sb)) || (rc = dalloc(&s->ro_cfl, nck * P))) return rc;
    s->ro_cap = nck;
  }
  if ((rc = upload_com_weights(s))) return rc;
  const int64_t step0 = s->step;
  for (int64_t c = 0; c < nck; ++c) {
    VX_CUDA(cudaMemcpyAsync(s->ro_ckpt + c * sb, cur_state(s), 4 * sb, cudaMemcpyDeviceToDevice, st));
    VX_CUDA(cudaMemcpyAsync(s->ro_cfl + c * P, s->flags, N, cudaMemcpyDeviceToDevice, st));
    if ((rc = vx_step_async(s, std::min<int64_t>(K, n - c * K), stream))) return rc;
  }
  launch_com_travel(cur_state(s), s->ro_ckpt, P, s->cw, s->bstart, s->L.n_bodies, s->loss_d, st);
  VX_CUDA(cudaGetLastError());
  if (loss_body)
    VX_CUDA(cudaMemcpyAsync(loss_body, s->loss_d, 4 * (size_t)s->L.n_bodies, cudaMemcpyDeviceToHost, st));
  int32_t code;
  int64_t bs, bv;
  if ((rc = vx_get_status(s, stream, &code, &bs, &bv))) return rc;
  if (code == VX_ERR_UNSTABLE)
    return fail(code, "non-finite state at step " + std::to_string(bs) + ", voxel " + std::to_string(bv));
  s->ro_steps = n;
  s->ro_K = K;
  s->ro_step0 = step0;
  s->ro_gen = s->gen;
  return VX_OK;
}

int vx_rollout_backward(vx_sim* s, const float* w_body, float* grad_logE, float* grad_phase, void* stream) {
  const Range range("vx_rollout_backward");
  int rc = check_sim(s);
  if (rc) return rc;
  if (s->ro_steps == 0 || s->ro_gen != s->gen)
    return fail(VX_ERR_STATE, "no rollout recorded since the state or the model last changed");
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t N = s->L.N, P = s->pitch;
  const size_t sb = (size_t)NPLANE * P;
  const int64_t n = s->ro_steps, K = s->ro_K, nck = (n + K - 1) / K;
  if (s->ro_seg_cap < K + 1) {
    dfree(s->ro_seg);
    dfree(s->ro_sfl);
    dfree(s->ro_sfm);
    s->ro_seg_cap = 0;
    if ((rc = dalloc(&s->ro_seg, (K + 1) * sb)) || (rc = dalloc(&s->ro_sfl, (K + 1) * P)) ||
        (rc = dalloc(&s->ro_sfm, K * 6 * P)))
      return rc;
    s->ro_seg_cap = (int)(K + 1);
  }
  if (!s->adj && (rc = dalloc(&s->adj, adjoint_work_floats(P)))) return rc;
  const size_t asm_bytes = adj_tile_smem_bytes(s->tile_max, (int)s->L.palette.size());
  if (asm_bytes != s->adj_smem) {
    if (prepare_adj_tile(s->tile_max, asm_bytes) != 0)
      return fail(VX_ERR_CUDA, "adjoint kernel needs " + std::to_string(asm_bytes) + " bytes of shared memory");
    s->adj_smem = asm_bytes;
  }
  std::vector<float> wb(s->L.n_bodies, 1.f);
  if (w_body) wb.assign(w_body, w_body + s->L.n_bodies);
  VX_CUDA(cudaMemcpy(s->wb_d, wb.data(), 4 * wb.size(), cudaMemcpyHostToDevice));
  int lam_cur = 0;
  AdjArgs J = adjoint_args(s->adj, P, lam_cur);
  launch_seed_adjoint(const_cast<float*>(J.lam_in), P, (int)N, s->cw, s->body, s->wb_d, st);
  VX_CUDA(cudaMemsetAsync(J.grad_logE, 0, 4 * 2 * (size_t)P, st));  // grad_logE, grad_phase
  for (int64_t c = nck - 1; c >= 0; --c) {
    const int64_t len = std::min<int64_t>(K, n - c * K);
    const int64_t sc0 = s->ro_step0 + c * K;
    // recompute the segment's states, flags and bond sums from its checkpoint
    VX_CUDA(cudaMemcpyAsync(s->ro_seg, s->ro_ckpt + c * sb, 4 * sb, cudaMemcpyDeviceToDevice, st));
    VX_CUDA(cudaMemcpyAsync(s->ro_sfl, s->ro_cfl + c * P, N, cudaMemcpyDeviceToDevice, st));
    for (int64_t j = 0; j < len; ++j) {
      VX_CUDA(cudaMemcpyAsync(s->ro_sfl + (j + 1) * P, s->ro_sfl + j * P, N, cudaMemcpyDeviceToDevice, st));
      StepArgs A = step_args(s);
      A.st_in = s->ro_seg + j * sb;
      A.st_out = s->ro_seg + (j + 1) * sb;
      A.flags = s->ro_sfl + (j + 1) * P;
      A.fm_out = s->ro_sfm + j * 6 * P;
      A.step = sc0 + j;
      A.act_w = act_phase(s, A.step);
      if ((rc = launch_form_step(s, A, st))) return rc;
    }
    // reverse steps
    for (int64_t j = len - 1; j >= 0; --j) {
      StepArgs A = step_args(s);
      A.st_in = s->ro_seg + j * sb;
      A.st_out = nullptr;
      A.flags = s->ro_sfl + j * P;
      A.step = sc0 + j;
      A.act_w = act_phase(s, A.step);
      AdjArgs Jj = adjoint_args(s->adj, P, lam_cur);
      Jj.fm = s->ro_sfm + j * 6 * P;
      launch_adjoint_step(A, Jj, s->tile_max, s->adj_smem, st);
      lam_cur ^= 1;
    }
  }
  if (grad_logE) launch_to_canonical(J.grad_logE, s->iperm, (int)N, grad_logE, st);
  if (grad_phase) launch_to_canonical(J.grad_phase, s->iperm, (int)N, grad_phase, st);
  VX_CUDA(cudaGetLastError());
  VX_CUDA(cudaStreamSynchronize(st));
  return VX_OK;
}

int vx_graph_capture(vx_sim* s, int64_t n, void* stream) {
  (void)stream;
  int rc = check_sim(s);
  if (rc) return rc;
  if (n < 1 || n > INT32_MAX) return fail(VX_ERR_ARG, "n_steps must be in [1, 2^31)");
  if (s->group_voxels == 0) return fail(VX_ERR_STATE, "graph capture takes the batched form (vx_set_batching)");
  if (s->collide_on) return fail(VX_ERR_STATE, "the batched form has no voxel-voxel collisions");
  const bool res = is_resident(s->group_voxels);
  if (res) {
    if ((rc = ensure_resident(s))) return rc;  // before step_args: it may allocate the neighbour planes
    if (s->res_ok != 1) return fail(VX_ERR_STATE, "the resident form does not fit this lattice");
  }
  StepArgs A = step_args(s);
  if (!res) {
    if ((rc = ensure_pipe(s, A))) return rc;
    if ((int64_t)s->B.cta_start.size() != (int64_t)s->pipe_grid + 1 && (rc = build_schedule(s))) return rc;
  }
  if (!s->ctr_d && (rc = dalloc(&s->ctr_d, 2))) return rc;
  BatchArgs Bt = batch_args(s, n);
  Bt.ctr = s->ctr_d;
  ResArgs R = res_args(s, n);
  R.ctr = s->ctr_d;
  cudaStream_t cs;
  VX_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    if (res) e = launch_resident(A, R, s->res_grid, s->res_C, s->res_threads, s->res_smem, s->res_per_voxel, cs);
    else launch_batched(A, Bt, s->tile_max, s->pipe_smem, s->pipe_grid, cs);
    const cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) return fail(VX_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  if (s->gexec) cudaGraphExecDestroy(s->gexec);
  s->gexec = ge;
  s->g_n = n;
  s->g_cfg = s->cfg;
  return VX_OK;
}

int vx_graph_launch(vx_sim* s, void* stream) {
  int rc = check_sim(s);
  if (rc) return rc;
  if (!s->gexec || s->g_cfg != s->cfg)
    return fail(VX_ERR_STATE, "no graph captured for the current model and step form");
  ++s->gen;
  cudaStream_t st = (cudaStream_t)stream;
  s->ctr_h[0] = s->step;
  s->ctr_h[1] = s->cur;
  VX_CUDA(cudaMemcpyAsync(s->ctr_d, s->ctr_h, sizeof(s->ctr_h), cudaMemcpyHostToDevice, st));
  VX_CUDA(cudaGraphLaunch(s->gexec, st));
  s->cur ^= (int)(s->g_n & 1);
  s->step += s->g_n;
  return VX_OK;
}

int vx_autotune_batching(vx_sim* s, int32_t sample_steps, int32_t* tile_max_out, int64_t* group_voxels_out,
                         double* rate_out, void* stream) {
  int rc = check_sim(s);
  if (rc) return rc;
  if (sample_steps < 1) return fail(VX_ERR_ARG, "sample_steps must be >= 1");
  if (s->collide_on) return fail(VX_ERR_STATE, "the batched form has no voxel-voxel collisions");
  cudaStream_t st = (cudaStream_t)stream;
  const TuneKey key = tune_key(s);
  TuneVal best{0, 0, 0.0};
  bool cached = false;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) { best = it->second; cached = true; }
  }
  if (!cached) {
    // time every candidate from the same state, then put the state back
    const int64_t N = s->L.N, P = s->pitch;
    const size_t sb = (size_t)NPLANE * P;
    float* save = nullptr;
    uint8_t* save_fl = nullptr;
    if ((rc = dalloc(&save, sb)) || (rc = dalloc(&save_fl, N))) { dfree(save); return rc; }
    const int64_t step0 = s->step;
    const int cur0 = s->cur;
    auto restore = [&]() -> int {
      s->cur = cur0;
      s->step = step0;
      VX_CUDA(cudaMemcpyAsync(cur_state(s), save, 4 * sb, cudaMemcpyDeviceToDevice, st));
      VX_CUDA(cudaMemcpyAsync(s->flags, save_fl, N, cudaMemcpyDeviceToDevice, st));
      return VX_OK;
    };
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto run = [&]() -> int {
      VX_CUDA(cudaMemcpyAsync(save, cur_state(s), 4 * sb, cudaMemcpyDeviceToDevice, st));
      VX_CUDA(cudaMemcpyAsync(save_fl, s->flags, N, cudaMemcpyDeviceToDevice, st));
      const int tiles[2] = {128, 256};
      const int64_t groups[6] = {0, 1024, 4096, 16384, 65536, VX_GROUPS_RESIDENT};
      int r;
      if ((r = ensure_resident(s))) return r;
      const bool res_possible = s->res_ok == 1;
      for (int tm : tiles)
        for (int64_t gv : groups) {
          if (gv == VX_GROUPS_RESIDENT && (!res_possible || tm != 256)) continue;  // no tiles in that form
          if ((r = vx_set_step_form(s, VX_FORM_PIPELINED, tm)) || (r = vx_set_batching(s, gv))) return r;
          if ((r = vx_step_async(s, 2, st)) || (r = restore())) return r;  // warm-up (prepares kernels)
          VX_CUDA(cudaEventRecord(e0, st));
          if ((r = vx_step_async(s, sample_steps, st))) return r;
          VX_CUDA(cudaEventRecord(e1, st));
          VX_CUDA(cudaEventSynchronize(e1));
          float ms = 0.f;
          VX_CUDA(cudaEventElapsedTime(&ms, e0, e1));
          int32_t code;
          int64_t bs, bv;
          if ((r = vx_get_status(s, st, &code, &bs, &bv))) return r;
          if ((r = restore())) return r;
          if (code != VX_OK) return fail(code, "autotuning sample became unstable");
          const double rate = (double)N * sample_steps / (1e-3 * ms);
          if (rate > best.rate) best = TuneVal{tm, gv, rate};
        }
      return VX_OK;
    };
    rc = run();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(st);
    dfree(save);
    dfree(save_fl);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = best;
  }
  if ((rc = vx_set_step_form(s, VX_FORM_PIPELINED, best.tile_max))) return rc;
  if ((rc = vx_set_batching(s, best.group_voxels))) {
    // a cached resident choice from a lattice of the same size class whose
    // largest body fitted a cluster: per-step launches instead
    if (!is_resident(best.group_voxels) || (rc = vx_set_batching(s, 0))) return rc;
    best.group_voxels = 0;
  }
  if (tile_max_out) *tile_max_out = best.tile_max;
  if (group_voxels_out) *group_voxels_out = best.group_voxels;
  if (rate_out) *rate_out = best.rate;
  return VX_OK;
}

int vx_audit(vx_sim* s, double* out, void* stream) {
  int rc = check_sim(s);
  if (rc) return rc;
  if (!out) return fail(VX_ERR_ARG, "out is NULL");
  if ((rc = ensure_nbr(s))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const Lattice& L = s->L;
  const int nb = L.n_bodies, nm = (int)L.palette.size(), np = audit_partials((int)L.N);
  const size_t n_in = 3 * (size_t)nb + 4 * (size_t)nm;
  const size_t n_all = n_in + 10 * (size_t)np + 10;
  dfree(s->aud);
  if ((rc = dalloc(&s->aud, n_all))) return rc;
  std::vector<double> h(n_in);
  for (int b = 0; b < nb; ++b)
    for (int a = 0; a < 3; ++a) h[3 * b + a] = (double)L.origin[3 * b + a];
  const double l = (double)L.l;
  double* hm = h.data() + 3 * nb;
  for (int m = 0; m < nm; ++m) {
    const vx_material& p = L.palette[m];
    const double mass = (double)p.rho * l * l * l;
    hm[m] = (double)p.E;
    hm[nm + m] = 1.0 / (2.0 * (1.0 + (double)p.nu));
    hm[2 * nm + m] = mass;
    hm[3 * nm + m] = mass * l * l / 6.0;
  }
  VX_CUDA(cudaMemcpy(s->aud, h.data(), n_in * sizeof(double), cudaMemcpyHostToDevice));
  AuditArgs U;
  U.l = l;
  U.gz = (double)s->gz;
  U.origin = s->aud;
  U.E = s->aud + 3 * nb;
  U.g_ratio = U.E + nm;
  U.mass = U.E + 2 * nm;
  U.inertia = U.E + 3 * nm;
  StepArgs A = step_args(s);
  A.nbr = s->nbr;
  A.act_w = act_phase(s, s->step);
  double* partial = s->aud + n_in;
  double* res = partial + 10 * (size_t)np;
  launch_audit(A, U, partial, res, st);
  VX_CUDA(cudaGetLastError());
  VX_CUDA(cudaMemcpyAsync(out, res, 10 * sizeof(double), cudaMemcpyDeviceToHost, st));
  VX_CUDA(cudaStreamSynchronize(st));
  return VX_OK;
}

int vx_set_multistep(vx_sim* s, int32_t on) {
  if (s) ++s->cfg;
  int rc = check_sim(s);
  if (rc) return rc;
  if (on < 0 || on > 2) return fail(VX_ERR_ARG, "multistep must be 0, 1 or 2");
  s->multistep = on;
  return VX_OK;
}

int vx_set_barrier_limits(vx_sim* s, int64_t max_spins, int32_t phantom_ctas) {
  int rc = check_sim(s);
  if (rc) return rc;
  if (max_spins < 0 || phantom_ctas < 0) return fail(VX_ERR_ARG, "limits must be >= 0");
  s->bar_spins = max_spins == 0 ? (1ll << 24) : max_spins;
  s->bar_extra = phantom_ctas;
  return VX_OK;
}

int vx_relax(vx_sim* s, int64_t max_steps, double v_tol, int32_t check_every, int64_t* steps_taken,
             double* max_speed, int32_t* converged, void* stream) {
  int rc = check_sim(s);
  if (rc) return rc;
  if (max_steps < 0 || check_every < 1 || !(v_tol >= 0.0))
    return fail(VX_ERR_ARG, "max_steps >= 0, check_every >= 1 and v_tol >= 0 are required");
  cudaStream_t st = (cudaStream_t)stream;
  if (!s->vmax_d && (rc = dalloc(&s->vmax_d, 1))) return rc;
  int64_t done = 0;
  float vmax = 0.f;
  bool ok = false;
  for (;;) {
    VX_CUDA(cudaMemsetAsync(s->vmax_d, 0, sizeof(unsigned), st));
    launch_max_speed(cur_state(s), s->pitch, (int)s->L.N, s->vmax_d, st);
    unsigned bits = 0;
    VX_CUDA(cudaMemcpyAsync(&bits, s->vmax_d, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    int32_t code;
    int64_t bs, bv;
    if ((rc = vx_get_status(s, stream, &code, &bs, &bv))) return rc;  // waits for the stream
    if (code == VX_ERR_UNSTABLE)
      return fail(code, "non-finite state at step " + std::to_string(bs) + ", voxel " + std::to_string(bv));
    std::memcpy(&vmax, &bits, sizeof(vmax));
    if (done > 0 && (double)vmax <= v_tol) { ok = true; break; }
    if (done >= max_steps) break;
    const int64_t n = std::min<int64_t>(check_every, max_steps - done);
    if ((rc = vx_step_async(s, n, stream))) return rc;
    done += n;
  }
  if (steps_taken) *steps_taken = done;
  if (max_speed) *max_speed = (double)vmax;
  if (converged) *converged = ok ? 1 : 0;
  return VX_OK;
}

int vx_set_collision_scheme(vx_sim* s, int32_t all_voxels, int32_t every_step) {
  if (s) { ++s->gen; ++s->cfg; }
  int rc = check_sim(s);
  if (rc) return rc;
  const int all = all_voxels ? 1 : 0;
  if (all != s->coll_all && s->coll_alloc) {
    VX_CUDA(cudaDeviceSynchronize());
    free_collisions(s);
  }
  s->coll_all = all;
  s->coll_every = every_step ? 1 : 0;
  if (s->collide_on) {
    if ((rc = force_rebuild(s, 0))) return rc;
    VX_CUDA(cudaDeviceSynchronize());
  }
  return VX_OK;
}

}  // extern "C"

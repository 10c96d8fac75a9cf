// Launch wrappers of the library's kernels (host-callable).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "vx_dev.cuh"

namespace vx {

// Raises a kernel's dynamic shared memory limit to the most the device allows
// next to the kernel's static shared memory.  Setting the largest value (not
// the size one simulator needs) means simulators of different sizes in one
// process never lower each other's limit.  Fails if `need` is above it.
template <class F> inline cudaError_t allow_smem(F* kernel, size_t need) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa;
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, (const void*)kernel);
  if (e != cudaSuccess) return e;
  const int allowed = optin - (int)fa.sharedSizeBytes;
  if (allowed < 0 || (size_t)allowed < need) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute((const void*)kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, allowed);
}

struct CollideArgs {
  int S;                  // surface voxels
  int n_bodies;
  int H;                  // hash buckets (power of two)
  int K;                  // quantisation: offset * 2^K
  int64_t Q;              // quantisation: lattice step rint(l 2^K)
  int64_t ostride_v;      // offsets: component a of voxel v at st[v * ostride_v + a * ostride_a]
  int64_t ostride_a;
  float threshold;        // horizon accumulator threshold [m]
  const float* st;        // offsets (see the strides)
  const int32_t* surf;    // surface voxel list (canonical, ascending)
  const uint32_t* lat;
  const int32_t* body;    // or nullptr
  const float* dt_body;
  int64_t* xq;            // 3 planes of S
  int4* cell;             // S: integer cell (edge = horizon) of each searched voxel
  uint32_t* bucket;       // S
  uint32_t* hcount;       // H
  uint32_t* hcursor;      // H
  uint32_t* hstart;       // H + 1
  uint32_t* bsum;         // ceil(H / 1024)
  int32_t* sorted;        // S
  // the searched voxels in bucket order (written by the scatter, read by the
  // query as contiguous runs): cell and searched index (x, y, z, t), the
  // quantised coordinates (3 planes of S) and (voxel, lattice word, body, 0)
  int4* scell;
  int64_t* sxq;
  int4* sinf;
  int32_t* ccount;        // S
  int32_t* vcnt;          // per voxel (internal order): the same counts for the step, or nullptr
  int32_t* cand;          // S x kCandCap
  float* acc;             // per body
  unsigned* vmax_bits;    // per body
  int* flag;              // per body rebuild flag
  int* any;               // any body flagged
  long long* n_rebuilds;
  int* status;
  const int64_t* qorg;    // shared world: quantised body origins (3 per body), else nullptr
  unsigned* bar;          // grid barrier words of the rebuild launch (zero at setup)
  long long spins;        // barrier wait budget (units of 128 SM cycles)
  unsigned extra = 0;     // CTAs the rebuild launch's barriers wait for beyond the grid (fault injection; 0)
};

// Error code of a device status word (the first set bit in the order
// unstable, timeout, capacity, argument), VX_OK when none is set.
int status_code(int bits);
// the rebuild launch uses at most this many CTAs (bsum holds one entry per CTA)
constexpr int kRebuildMaxGrid = 1024;

// form 0: fused tile kernel (tile_max threads per CTA, smem bytes of dynamic
// shared memory); form 1: two-pass bond_pass + voxel_pass.
void launch_step(const StepArgs& A, int form, int tile_max, size_t smem, cudaStream_t s);
size_t fused_smem_bytes(int tile_max, int n_mats, bool lut);
// Raises the fused kernel's dynamic shared memory limit; 0 on success.
int prepare_fused(int tile_max, size_t smem);
// Pipelined persistent form: shared memory for the optional per-voxel arrays
// in use, kernel preparation (returns the persistent grid) and launch.
size_t pipe_smem_bytes(int tile_max, bool ph, bool le, bool body, bool fext, bool col, int n_mats, bool lut);
int prepare_pipe(int tile_max, size_t smem, int* grid);
void launch_pipe(const StepArgs& A, int tile_max, size_t smem, int grid, cudaStream_t s);

// Batched multi-step form (independent bodies, no collisions).
struct BatchArgs {
  const int32_t* cta_start;    // grid + 1
  const int32_t* cta_groups;
  const int32_t* group_tiles;  // 2 per group
  float* buf0;                 // the two state buffers
  float* buf1;
  int cur0;                    // buffer holding the state at step0
  int n_steps;
  int64_t step0;
  int64_t act_P;
  float act_c;                 // fl(2 pi / act_P)
  const int64_t* ctr;          // device (step0, cur0) read at launch instead, or nullptr
};
int prepare_batched(int tile_max, size_t smem);

// Multi-step form: one cooperative launch of min(n_tiles, co-resident CTAs)
// CTAs runs n_steps with a bounded grid barrier (bar: 2 device words, zero
// at launch) between steps.
struct MultiArgs {
  float* buf0;                 // the two state buffers
  float* buf1;
  int cur0;                    // buffer holding the state at step0
  int n_steps;
  int64_t step0;
  int64_t act_P;
  float act_c;                 // fl(2 pi / act_P)
  const int64_t* ctr;          // device (step0, cur0) read at launch instead, or nullptr
  unsigned* bar;               // barrier count and generation
  long long spins;             // wait budget of one barrier (units of 128 SM cycles)
  unsigned extra;              // CTAs the barrier waits for beyond the grid (fault injection; 0)
  // collisions between the steps: after each step the horizon (or, with
  // every_step, a forced rebuild) and, when a body is flagged, the rebuild
  // phases on the same grid and barrier (coll.st is set per step)
  int collide, every_step;
  CollideArgs coll;
};
int prepare_multi(int tile_max, size_t smem, int n_tiles, int* grid, int* co_resident);

// Shared-memory-resident form: groups of whole bodies, each kept in the
// shared memory of one cluster of C CTAs (kResThreads threads, up to `cap`
// voxels each) for all n_steps of a launch; no voxel-voxel collisions.
constexpr int kResThreads = 512;
struct ResArgs {
  const int32_t* grp_start;    // n_groups + 1 internal voxel offsets of the groups
  const int32_t* cl_start;     // n_clusters + 1 offsets into cl_groups
  const int32_t* cl_groups;    // group indices, per cluster in processing order
  float* buf0;                 // the two state buffers
  float* buf1;
  int cur0;                    // buffer holding the state at step0
  int n_steps;
  int64_t step0;
  int64_t act_P;
  float act_c;                 // fl(2 pi / act_P)
  const int64_t* ctr;          // device (step0, cur0) read at launch instead, or nullptr
  int cap;                     // voxels per CTA slice (shared memory layout)
};
size_t res_smem_bytes(int cap, bool fext, int n_mats, bool lut);
// Raises the kernel's limits for clusters of C CTAs of `threads` threads
// (at most kResThreads) and returns how many such clusters can be resident
// at once; 0 on success.  per_voxel: one thread per voxel in the bond phase
// (its own +x, +y, +z bonds, rotation matrix once), else one thread per bond.
int prepare_resident(int C, int threads, size_t smem, bool fext, bool per_voxel, int* max_clusters);
// Needs A.nbr (internal neighbour planes); grid is a multiple of C.
cudaError_t launch_resident(const StepArgs& A, const ResArgs& R, int grid, int C, int threads, size_t smem,
                            bool per_voxel, cudaStream_t s);
cudaError_t launch_multi(const StepArgs& A, const MultiArgs& M, int tile_max, size_t smem, int grid, cudaStream_t s);
void launch_batched(const StepArgs& A, const BatchArgs& B, int tile_max, size_t smem, int grid, cudaStream_t s);
void launch_horizon(const CollideArgs& C, cudaStream_t s);
// bond_pass of the two-pass form alone (bond results into A.bf)
void launch_bond_pass(const StepArgs& A, cudaStream_t s);

// Adjoint form: buffers of one reverse step (pitch floats per plane; all
// but fm live in one work array laid out by adjoint_args).
struct AdjArgs {
  const float* lam_in;   // adjoint of the state at step n + 1 (state layout)
  float* lam_out;        // adjoint of the state at step n (state layout)
  const float* fm;       // 6 planes: bond force and moment sums at step n (recorded)
  float* gfm;            // 6 planes: their adjoints
  float* gdir;           // 2 planes: the voxel's own dL/dE and dL/d(thermal strain)
  float* grad_logE;      // accumulated dL/d(log E), internal order
  float* grad_phase;     // accumulated dL/d(phase), internal order
};
int64_t adjoint_work_floats(int64_t pitch);
// lam_cur: which of the two adjoint state buffers holds lam_{n+1}
AdjArgs adjoint_args(float* work, int64_t pitch, int lam_cur);
size_t adj_tile_smem_bytes(int tile_max, int n_mats);
int prepare_adj_tile(int tile_max, size_t smem);
// One reverse step: A.st_in = S_n, A.flags = flags at step n, A.act_w and
// A.step of step n, the fused form's tile arrays; J.fm = bond sums at step n.
void launch_adjoint_step(const StepArgs& A, const AdjArgs& J, int tile_max, size_t smem, cudaStream_t s);
// FP64 audit (momentum, angular momentum, energies); needs A.nbr.  The
// per-material and per-body values are FP64 copies of the host's inputs.
struct AuditArgs {
  double l, gz;
  const double* origin;   // 3 per body
  const double* E;        // per material: E, G / E, rho l^3, m l^2 / 6
  const double* g_ratio;
  const double* mass;
  const double* inertia;
};
int audit_partials(int N);
// out[10] (device): P (3), L about the origin (3), KE linear, KE rotational,
// U elastic, U gravity; partial: audit_partials(N) x 10 doubles
void launch_audit(const StepArgs& A, const AuditArgs& U, double* partial, double* out, cudaStream_t s);

// Stable timestep reduction (FP32, set-up work).  Chunks of at most
// kDtChunk voxels, one per CTA, each inside one body's internal range:
// (v0, v1, body, 0).  w2 [n_bodies] holds zero at launch and receives, as
// the bits of a float, the body's largest w^2 [1/s^2].
constexpr int kDtThreads = 256;
constexpr int kDtChunk = 8 * kDtThreads;
struct DtArgs {
  int n_chunks;
  int64_t N;
  float l;                // voxel size [m]
  const uint8_t* mat;     // per voxel (internal order)
  const float* logE;      // per voxel natural-log modulus overriding the palette, or nullptr
  const int32_t* nbr;     // 6 planes (-x,+x,-y,+y,-z,+z), internal indices, -1: no bond
  const DevMat* mats;     // E and m = rho l^3 of every material
  const int4* chunks;
  unsigned* w2;
};
void launch_stable_w2(const DtArgs& D, cudaStream_t s);

void launch_seed_adjoint(float* lam, int64_t pitch, int N, const float* cw, const int32_t* body,
                         const float* w_body, cudaStream_t s);
// loss[b] = sum over the body's internal range of cw (x(end) - x(start))
void launch_com_travel(const float* st1, const float* st0, int64_t pitch, const float* cw, const int32_t* bstart,
                       int n_bodies, float* loss, cudaStream_t s);
void launch_to_canonical(const float* g, const int32_t* iperm, int N, float* out, cudaStream_t s);
void launch_rebuild(const CollideArgs& C, cudaStream_t s);
// A write of the state as motion for the collision horizon: every body's
// accumulator grows by twice its largest written displacement dmax (float
// bits, zeroed here); bodies at the threshold are flagged (world: one
// accumulator, every body flagged), and so is every body when the status
// word holds a timed-out or overflowed rebuild.
void launch_write_horizon(const CollideArgs& C, unsigned* dmax, int world, cudaStream_t s);
void launch_flag_all(const CollideArgs& C, cudaStream_t s);

// internal-order device state <-> interleaved canonical-order caller layout
// (offset[N][3], quat[N][4], vel[N][3], angvel[N][3], flags[N]); iperm maps
// canonical to internal indices; any destination/source pointer may be null
void launch_pack_state(const float* st, int64_t pitch, int N, const int32_t* iperm, const uint8_t* flags,
                       float* off, float* quat, float* vel, float* angvel, uint8_t* fl, cudaStream_t s);
// The unpacking takes perm (internal -> canonical) instead of iperm.  With
// dmax (per body, float bits, zero at launch) the largest distance between
// written and current offsets is recorded per body (body: per voxel,
// internal order, or nullptr for one body).
void launch_unpack_state(float* st, int64_t pitch, int N, const int32_t* perm, uint8_t* flags, const float* off,
                         const float* quat, const float* vel, const float* angvel, const uint8_t* fl,
                         cudaStream_t s, const int32_t* body = nullptr, unsigned* dmax = nullptr);
// atomic max of |v| over the voxels into *out (float bits; zero it first)
void launch_max_speed(const float* st, int64_t pitch, int N, unsigned* out, cudaStream_t s);
// rest state: zero offsets, identity quaternions, v0 for non-fixed voxels
void launch_reset_state(float* st, int64_t pitch, int N, uint8_t* flags, float v0x, float v0y, float v0z,
                        cudaStream_t s);
void launch_set_velocity(float* st, int64_t pitch, int N, const uint8_t* flags, float vx, float vy, float vz,
                         cudaStream_t s);

}  // namespace vx

// Host-side lattice description shared by the library's translation units.
// Pure C++ (no CUDA): the lattice build, timestep and region selection run on
// the host once per create / parameter change.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "vx.h"

namespace vx {

// Packed lattice coordinate of a voxel: i | j << 11 | k << 22.
inline uint32_t pack_ijk(int i, int j, int k) { return (uint32_t)i | ((uint32_t)j << 11) | ((uint32_t)k << 22); }
inline int lat_i(uint32_t p) { return (int)(p & 2047u); }
inline int lat_j(uint32_t p) { return (int)((p >> 11) & 2047u); }
inline int lat_k(uint32_t p) { return (int)(p >> 22); }

struct Lattice {
  int n_bodies = 0;
  std::vector<int32_t> dims;        // 3 per body
  float l = 0.f;
  std::vector<vx_material> palette;
  std::vector<float> origin;        // 3 per body
  int64_t N = 0, n_bonds = 0, n_surface = 0;
  std::vector<int32_t> body;        // per voxel
  std::vector<uint32_t> lat;        // per voxel, packed (i, j, k) within its body
  std::vector<uint8_t> mat;         // per voxel, 0-based palette index
  std::vector<int32_t> nbr;         // 6 planes of N: -x,+x,-y,+y,-z,+z neighbour or -1
  std::vector<int32_t> surf_list;   // canonical indices of surface voxels, ascending
  std::vector<int32_t> body_first;  // n_bodies + 1
};

// Validates the description and fills the lattice.  Returns VX_OK or an
// error code with a message in err.
int build_lattice(const vx_desc* d, Lattice& L, std::string& err);

// Per-body stable timestep (paper Sec 2.1.4) in double.
void stable_dt(const Lattice& L, const float* logE, float dt_factor, std::vector<double>& dt);

// Voxels touching a region given in workspace fractions (paper App. B).
int64_t region_mask(const Lattice& L, int body, const float loc[3], const float size[3], uint8_t* mask);

// Records the message vx_last_error() returns on this thread; returns code.
int set_error(int code, const std::string& msg);

// Collision quantisation: 2^K <= 65536 / l < 2^(K+1), Q = rint(l 2^K).
void quant_params(float l, int* K, int64_t* Q);

// Internal (device) voxel order and the tiles of the fused step kernel.
//
// Voxels are grouped into 4x4x4-site bricks; bricks of a body follow a 3-D
// Morton curve and voxels inside a brick follow the site order.  The fused
// kernel stages a tile plus its halo (face neighbours outside the tile) in
// shared memory.  Tiles are runs of tile_max consecutive voxels in this order
// (shorter only where owned + halo would exceed the staging limit).  Each
// owned voxel evaluates its own +x, +y, +z bonds (partner slots in `plus`);
// bonds whose negative-side voxel lies in the halo form the tile's short
// `halo_bonds` list.
struct Tiling {
  int tile_max = 0;
  int max_local = 0;             // max over tiles of owned + halo voxels
  int max_halo_bonds = 0;        // max over tiles of bonds entering from the halo (<= local_max)
  std::vector<int32_t> perm;     // internal -> canonical
  std::vector<int32_t> iperm;    // canonical -> internal
  std::vector<int32_t> tile_a;   // 4 per tile: v0, n_owned, halo start, n_halo
  std::vector<int32_t> tile_b;   // 4 per tile: halo-bond list start, end, 0, 0
  std::vector<int32_t> halo;     // internal voxel indices
  std::vector<uint16_t> plus;    // 3 planes of N: staging slot of the +a neighbour, 0xFFFF if none
  std::vector<uint32_t> halo_bonds;  // slot of voxel 1 | slot of voxel 2 << 12 | axis << 24
  std::vector<uint8_t> mask;     // per internal voxel: bit 2a (-a) / 2a+1 (+a) bond exists
  // Fixed-stride copies for the pipelined kernel: per tile 8 ints
  // (v0, n_owned, n_halo, halo-bond start, n_halo_bonds, 0, 0, 0) and the
  // tile's halo indices at halo_fixed[t * halo_stride + j].
  int halo_stride = 0;
  std::vector<int32_t> tile_desc;
  std::vector<int32_t> halo_fixed;
  int64_t n_tiles() const { return (int64_t)tile_a.size() / 4; }
  int64_t n_tile_bonds() const;  // bonds evaluated over all tiles
};

// Local slots must stay below 4096 (12-bit packing).
constexpr int kMaxLocal = 4095;

// local_max: largest owned + halo set, and largest list of bonds entering
// from the halo, a tile may stage (shared memory bound); tiles are shortened
// until both fit.  breaks (optional, ascending internal
// voxel indices): no tile crosses one.
int build_tiling(const Lattice& L, int tile_max, int local_max, Tiling& T, std::string& err,
                 const std::vector<int64_t>* breaks = nullptr);

// Batched schedule: consecutive bodies grouped to about group_voxels voxels
// (a body larger than that is its own group), groups dealt to n_ctas
// persistent CTAs longest first onto the least loaded CTA.  A group is a
// voxel range [v0, v1) in internal order; its tiles are [t0, t1).
struct Batch {
  std::vector<int64_t> group_start;   // n_groups + 1 voxel offsets (internal order)
  std::vector<int32_t> group_tiles;   // 2 per group: first tile, end tile
  std::vector<int32_t> cta_start;     // n_ctas + 1 offsets into cta_groups
  std::vector<int32_t> cta_groups;    // group indices, per CTA in processing order
  int64_t max_cta_voxels = 0;         // heaviest CTA's voxels (load balance)
};

// Resident schedule: consecutive whole bodies grouped while a group stays
// within max_group voxels, groups dealt longest first onto the least loaded
// of n_clusters clusters.  body_start: n_bodies + 1 internal voxel offsets.
// Returns false when a body alone exceeds max_group.
struct ResPlan {
  std::vector<int32_t> grp_start;     // n_groups + 1 internal voxel offsets
  std::vector<int32_t> cl_start;      // n_clusters + 1 offsets into cl_groups
  std::vector<int32_t> cl_groups;     // group indices, per cluster in processing order
  int64_t max_cluster_voxels = 0;
};
bool plan_resident(const std::vector<int64_t>& body_start, int64_t max_group, int n_clusters, ResPlan& P);

// Voxel offsets (internal order) where the groups of a batched schedule start.
std::vector<int64_t> batch_group_starts(const Lattice& L, int64_t group_voxels);
// Fills the tile ranges and the CTA assignment for groups starting at `starts`.
void build_batch(const Tiling& T, const std::vector<int64_t>& starts, int64_t N, int n_ctas, Batch& B);

}  // namespace vx

// Host lattice build: compaction of the material grid into voxels, bond
// neighbours, surface voxels, per-body stable timestep and region selection.
#include "vx_host.h"

#include <algorithm>
#include <cmath>

namespace vx {

int build_lattice(const vx_desc* d, Lattice& L, std::string& err) {
  if (!d) { err = "desc is NULL"; return VX_ERR_ARG; }
  if (d->n_bodies < 1 || !d->dims || !d->grid || !d->palette) { err = "desc: missing bodies, dims, grid or palette"; return VX_ERR_ARG; }
  if (d->n_materials < 1 || d->n_materials > 255) { err = "desc: n_materials must be in [1, 255]"; return VX_ERR_ARG; }
  if (!(d->voxel_size > 0.f) || !std::isfinite(d->voxel_size)) { err = "desc: voxel_size must be positive"; return VX_ERR_ARG; }
  for (int m = 0; m < d->n_materials; ++m) {
    const vx_material& p = d->palette[m];
    if (!(p.E > 0.f) || !(p.rho > 0.f) || !(p.nu > -1.f && p.nu < 0.5f) || !(p.mu_s >= 0.f) || !(p.mu_k >= 0.f) ||
        !std::isfinite(p.cte) || !std::isfinite(p.E) || !std::isfinite(p.rho)) {
      err = "desc: material " + std::to_string(m) + " out of range (E>0, rho>0, -1<nu<0.5, mu>=0)";
      return VX_ERR_ARG;
    }
  }
  L = Lattice();
  L.n_bodies = d->n_bodies;
  L.l = d->voxel_size;
  L.palette.assign(d->palette, d->palette + d->n_materials);
  L.dims.assign(d->dims, d->dims + 3 * d->n_bodies);
  L.origin.assign(3 * (size_t)d->n_bodies, 0.f);
  if (d->origin) L.origin.assign(d->origin, d->origin + 3 * d->n_bodies);
  std::vector<size_t> site_off(d->n_bodies + 1, 0);
  for (int b = 0; b < d->n_bodies; ++b) {
    int nx = L.dims[3 * b], ny = L.dims[3 * b + 1], nz = L.dims[3 * b + 2];
    if (nx < 1 || ny < 1 || nz < 1 || nx > 2048 || ny > 2048 || nz > 1024) {
      err = "desc: body " + std::to_string(b) + " dims out of range (1..2048, 1..2048, 1..1024)";
      return VX_ERR_ARG;
    }
    site_off[b + 1] = site_off[b] + (size_t)nx * ny * nz;
  }
  // count and validate
  int64_t N = 0;
  for (size_t s = 0; s < site_off[d->n_bodies]; ++s) {
    uint8_t m = d->grid[s];
    if (m == 0) continue;
    if (m > d->n_materials) { err = "desc: grid references material " + std::to_string(m) + " beyond the palette"; return VX_ERR_ARG; }
    ++N;
  }
  if (N == 0) { err = "desc: lattice has no occupied site"; return VX_ERR_ARG; }
  if (N >= (int64_t)1 << 31) { err = "desc: too many voxels"; return VX_ERR_ARG; }
  L.N = N;
  L.body.resize(N); L.lat.resize(N); L.mat.resize(N);
  L.body_first.assign(d->n_bodies + 1, 0);
  // site -> voxel index, per body, built on the fly (one body at a time)
  int64_t v = 0;
  L.nbr.assign(6 * (size_t)N, -1);
  std::vector<int32_t> s2v;
  for (int b = 0; b < d->n_bodies; ++b) {
    int nx = L.dims[3 * b], ny = L.dims[3 * b + 1], nz = L.dims[3 * b + 2];
    const uint8_t* g = d->grid + site_off[b];
    s2v.assign((size_t)nx * ny * nz, -1);
    L.body_first[b] = (int32_t)v;
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
          size_t s = (size_t)i + (size_t)nx * ((size_t)j + (size_t)ny * k);
          if (!g[s]) continue;
          s2v[s] = (int32_t)v;
          L.body[v] = b; L.lat[v] = pack_ijk(i, j, k); L.mat[v] = (uint8_t)(g[s] - 1);
          ++v;
        }
    for (int64_t u = L.body_first[b]; u < v; ++u) {
      int c[3] = {lat_i(L.lat[u]), lat_j(L.lat[u]), lat_k(L.lat[u])};
      int n[3] = {nx, ny, nz};
      int occ = 0;
      for (int a = 0; a < 3; ++a)
        for (int sgn = 0; sgn < 2; ++sgn) {
          int cc[3] = {c[0], c[1], c[2]};
          cc[a] += sgn ? 1 : -1;
          int32_t w = -1;
          if (cc[a] >= 0 && cc[a] < n[a]) w = s2v[(size_t)cc[0] + (size_t)nx * ((size_t)cc[1] + (size_t)ny * cc[2])];
          L.nbr[(size_t)(2 * a + sgn) * N + u] = w;
          if (w >= 0) ++occ;
          if (w >= 0 && sgn) ++L.n_bonds;
        }
      if (occ < 6) L.surf_list.push_back((int32_t)u);
    }
  }
  L.body_first[d->n_bodies] = (int32_t)v;
  L.n_surface = (int64_t)L.surf_list.size();
  return VX_OK;
}

void stable_dt(const Lattice& L, const float* logE, float dt_factor, std::vector<double>& dt) {
  std::vector<double> wmax(L.n_bodies, 0.0);
  const double l = L.l;
  auto E_of = [&](int64_t v) { return logE ? std::exp((double)logE[v]) : (double)L.palette[L.mat[v]].E; };
  auto m_of = [&](int64_t v) { return (double)L.palette[L.mat[v]].rho * l * l * l; };
  for (int64_t v = 0; v < L.N; ++v) {
    int b = L.body[v];
    double Ev = E_of(v), mv = m_of(v);
    wmax[b] = std::max(wmax[b], std::sqrt(Ev * l / mv));   // voxel's own contact spring
    for (int a = 0; a < 3; ++a) {
      int32_t u = L.nbr[(size_t)(2 * a + 1) * L.N + v];
      if (u < 0) continue;
      double Eu = E_of(u);
      double Ec = 2.0 * Ev * Eu / (Ev + Eu);
      double k = Ec * l;  // a1 = E_c A / l with A = l^2
      wmax[b] = std::max(wmax[b], std::sqrt(k / std::min(mv, m_of(u))));
    }
  }
  dt.assign(L.n_bodies, 0.0);
  for (int b = 0; b < L.n_bodies; ++b)
    dt[b] = wmax[b] > 0.0 ? (double)dt_factor / (2.0 * M_PI * wmax[b]) : 0.0;
}

int64_t region_mask(const Lattice& L, int body, const float loc[3], const float size[3], uint8_t* mask) {
  int64_t cnt = 0;
  const int32_t* n = &L.dims[3 * body];
  for (int64_t v = 0; v < L.N; ++v) {
    bool in = L.body[v] == body;
    int c[3] = {lat_i(L.lat[v]), lat_j(L.lat[v]), lat_k(L.lat[v])};
    for (int a = 0; a < 3 && in; ++a) {
      double lo = (double)c[a] / n[a], hi = (double)(c[a] + 1) / n[a];
      double r0 = loc[a], r1 = (double)loc[a] + (double)size[a];
      if (hi < r0 || lo > r1) in = false;
    }
    mask[v] = in ? 1 : 0;
    cnt += in ? 1 : 0;
  }
  return cnt;
}

void quant_params(float l, int* K, int64_t* Q) {
  int e = 0;
  std::frexp(65536.0 / (double)l, &e);
  *K = e - 1;
  *Q = (int64_t)std::nearbyint(std::ldexp((double)l, *K));
}

static uint64_t spread3(uint32_t x) {
  uint64_t v = x & 0x1fffffu;
  v = (v | v << 32) & 0x1f00000000ffffull;
  v = (v | v << 16) & 0x1f0000ff0000ffull;
  v = (v | v << 8) & 0x100f00f00f00f00full;
  v = (v | v << 4) & 0x10c30c30c30c30c3ull;
  v = (v | v << 2) & 0x1249249249249249ull;
  return v;
}

int build_tiling(const Lattice& L, int tile_max, int local_max, Tiling& T, std::string& err,
                 const std::vector<int64_t>* breaks) {
  if (tile_max < 64 || tile_max > 1024) { err = "tile size must be in [64, 1024]"; return VX_ERR_ARG; }
  local_max = std::min(local_max, kMaxLocal);
  if (local_max < 160) { err = "local_max must be at least 160 (one brick and its halo)"; return VX_ERR_ARG; }
  T = Tiling();
  T.tile_max = tile_max;
  const int64_t N = L.N;
  // --- order: (body, Morton(brick), site in brick)
  std::vector<std::pair<uint64_t, int32_t>> key(N);
  for (int64_t v = 0; v < N; ++v) {
    uint32_t p = L.lat[v];
    int i = lat_i(p), j = lat_j(p), k = lat_k(p);
    uint64_t m = spread3((uint32_t)(i >> 2)) | spread3((uint32_t)(j >> 2)) << 1 | spread3((uint32_t)(k >> 2)) << 2;
    uint64_t site = (uint64_t)((i & 3) | (j & 3) << 2 | (k & 3) << 4);
    key[v] = {m << 6 | site, (int32_t)v};
  }
  // bodies are contiguous in canonical order: sort inside each body
  for (int b = 0; b < L.n_bodies; ++b)
    std::sort(key.begin() + L.body_first[b], key.begin() + L.body_first[b + 1]);
  T.perm.resize(N);
  T.iperm.resize(N);
  for (int64_t v = 0; v < N; ++v) { T.perm[v] = key[v].second; T.iperm[key[v].second] = (int32_t)v; }
  // internal neighbour of internal voxel v in slot s, or -1
  auto nb = [&](int64_t v, int s) -> int32_t {
    int32_t c = L.nbr[(size_t)s * N + T.perm[v]];
    return c < 0 ? -1 : T.iperm[c];
  };
  T.mask.assign(N, 0);
  for (int64_t v = 0; v < N; ++v)
    for (int s = 0; s < 6; ++s)
      if (nb(v, s) >= 0) T.mask[v] |= (uint8_t)(1u << s);
  // --- tiles: runs of tile_max consecutive voxels (shortened while the
  // staged set, owned + halo, exceeds local_max)
  T.plus.assign(3 * (size_t)N, 0xFFFFu);
  std::vector<int32_t> hl;
  int64_t v0 = 0;
  size_t nb_i = 0;
  while (v0 < N) {
    int64_t len = std::min<int64_t>(tile_max, N - v0);
    if (breaks) {
      while (nb_i < breaks->size() && (*breaks)[nb_i] <= v0) ++nb_i;
      if (nb_i < breaks->size()) len = std::min<int64_t>(len, (*breaks)[nb_i] - v0);
    }
    for (;;) {
      int64_t v1 = v0 + len;
      hl.clear();
      int64_t nhb = 0;  // bonds entering from the halo (negative-side voxel outside the run)
      for (int64_t v = v0; v < v1; ++v)
        for (int s = 0; s < 6; ++s) {
          int32_t u = nb(v, s);
          if (u >= 0 && (u < v0 || u >= v1)) {
            hl.push_back(u);
            if ((s & 1) == 0) ++nhb;
          }
        }
      std::sort(hl.begin(), hl.end());
      hl.erase(std::unique(hl.begin(), hl.end()), hl.end());
      int64_t nl = len + (int64_t)hl.size();
      // both the staged set and the halo-bond list live in local_max slots
      const bool fits = nl <= local_max && nhb <= local_max;
      if (fits || len <= 32 || (breaks && len < 32)) {
        if (!fits) { err = "tile staging set too large"; return VX_ERR_ARG; }
        int32_t T0 = (int32_t)len;
        T.tile_a.insert(T.tile_a.end(), {(int32_t)v0, T0, (int32_t)T.halo.size(), (int32_t)hl.size()});
        auto local = [&](int32_t u) -> uint32_t {
          if (u >= v0 && u < v1) return (uint32_t)(u - v0);
          return (uint32_t)(T0 + (std::lower_bound(hl.begin(), hl.end(), u) - hl.begin()));
        };
        int32_t hb0 = (int32_t)T.halo_bonds.size();
        for (int64_t v = v0; v < v1; ++v)
          for (int a = 0; a < 3; ++a) {
            int32_t up = nb(v, 2 * a + 1);
            if (up >= 0) T.plus[(size_t)a * N + v] = (uint16_t)local(up);
            int32_t dn = nb(v, 2 * a);
            if (dn >= 0 && (dn < v0 || dn >= v1))
              T.halo_bonds.push_back(local(dn) | (uint32_t)(v - v0) << 12 | (uint32_t)a << 24);
          }
        T.tile_b.insert(T.tile_b.end(), {hb0, (int32_t)T.halo_bonds.size(), 0, 0});
        T.halo.insert(T.halo.end(), hl.begin(), hl.end());
        T.max_local = std::max<int>(T.max_local, (int)nl);
        T.max_halo_bonds = std::max<int>(T.max_halo_bonds, (int)nhb);
        v0 = v1;
        break;
      }
      len -= 32;
    }
  }
  // fixed-stride tile blocks
  T.halo_stride = local_max;
  const int64_t nt = T.n_tiles();
  T.tile_desc.assign(8 * (size_t)nt, 0);
  T.halo_fixed.assign((size_t)nt * T.halo_stride, -1);
  for (int64_t t = 0; t < nt; ++t) {
    const int32_t* a = &T.tile_a[4 * t];
    const int32_t* b = &T.tile_b[4 * t];
    int32_t* d = &T.tile_desc[8 * t];
    d[0] = a[0]; d[1] = a[1]; d[2] = a[3]; d[3] = b[0]; d[4] = b[1] - b[0];
    for (int32_t j = 0; j < a[3]; ++j) T.halo_fixed[(size_t)t * T.halo_stride + j] = T.halo[a[2] + j];
  }
  return VX_OK;
}

std::vector<int64_t> batch_group_starts(const Lattice& L, int64_t group_voxels) {
  // bodies are contiguous in internal order as in canonical order
  std::vector<int64_t> starts;
  int64_t acc = 0;
  for (int b = 0; b < L.n_bodies; ++b) {
    int64_t nb = L.body_first[b + 1] - L.body_first[b];
    if (starts.empty() || acc >= group_voxels || acc + nb > 2 * group_voxels) {
      starts.push_back(L.body_first[b]);
      acc = 0;
    }
    acc += nb;
  }
  return starts;
}

void build_batch(const Tiling& T, const std::vector<int64_t>& starts, int64_t N, int n_ctas, Batch& B) {
  B = Batch();
  const int64_t nt = T.n_tiles();
  B.group_start = starts;
  B.group_start.push_back(N);
  const size_t ng = starts.size();
  int32_t t = 0;
  for (size_t g = 0; g < ng; ++g) {
    int32_t t0 = t;
    while (t < nt && T.tile_a[4 * (size_t)t] < B.group_start[g + 1]) ++t;
    B.group_tiles.push_back(t0);
    B.group_tiles.push_back(t);
  }
  // longest processing time first onto the least loaded CTA
  std::vector<int32_t> order(ng);
  for (size_t g = 0; g < ng; ++g) order[g] = (int32_t)g;
  auto size_of = [&](int32_t g) { return B.group_start[g + 1] - B.group_start[g]; };
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return size_of(a) > size_of(b); });
  std::vector<int64_t> load(n_ctas, 0);
  std::vector<std::vector<int32_t>> lists(n_ctas);
  for (int32_t g : order) {
    int c = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    load[c] += size_of(g);
    lists[c].push_back(g);
  }
  B.cta_start.push_back(0);
  for (int c = 0; c < n_ctas; ++c) {
    B.cta_groups.insert(B.cta_groups.end(), lists[c].begin(), lists[c].end());
    B.cta_start.push_back((int32_t)B.cta_groups.size());
  }
  B.max_cta_voxels = *std::max_element(load.begin(), load.end());
}

bool plan_resident(const std::vector<int64_t>& body_start, int64_t max_group, int n_clusters, ResPlan& P) {
  P = ResPlan();
  const size_t nb = body_start.size() - 1;
  P.grp_start.push_back((int32_t)body_start[0]);
  int64_t cur = 0;
  for (size_t b = 0; b < nb; ++b) {
    const int64_t sz = body_start[b + 1] - body_start[b];
    if (sz > max_group) return false;
    if (cur > 0 && cur + sz > max_group) {
      P.grp_start.push_back((int32_t)body_start[b]);
      cur = 0;
    }
    cur += sz;
  }
  P.grp_start.push_back((int32_t)body_start[nb]);
  const size_t ng = P.grp_start.size() - 1;
  // longest processing time first onto the least loaded cluster
  std::vector<int32_t> order(ng);
  for (size_t g = 0; g < ng; ++g) order[g] = (int32_t)g;
  auto size_of = [&](int32_t g) { return (int64_t)P.grp_start[g + 1] - P.grp_start[g]; };
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return size_of(a) > size_of(b); });
  std::vector<int64_t> load(n_clusters, 0);
  std::vector<std::vector<int32_t>> lists(n_clusters);
  for (int32_t g : order) {
    const int c = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    load[c] += size_of(g);
    lists[c].push_back(g);
  }
  P.cl_start.push_back(0);
  for (int c = 0; c < n_clusters; ++c) {
    P.cl_groups.insert(P.cl_groups.end(), lists[c].begin(), lists[c].end());
    P.cl_start.push_back((int32_t)P.cl_groups.size());
  }
  P.max_cluster_voxels = *std::max_element(load.begin(), load.end());
  return true;
}

int64_t Tiling::n_tile_bonds() const {
  int64_t n = (int64_t)halo_bonds.size();
  for (uint16_t p : plus) n += p != 0xFFFFu;
  return n;
}

}  // namespace vx

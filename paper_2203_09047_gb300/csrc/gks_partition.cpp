// Domain decomposition of a mesh for several ranks (one process per GPU): a partition of the
// cells into contiguous ranges of the Morton order of their vertex means, whose sizes differ by
// at most one cell, and for each rank the halo its residual needs and the lists of cells it sends to the
// others. The residual of an owned cell i reads the reconstruction polynomials of i and of its
// face neighbours, and a polynomial reads the cell's big stencil (with every sub-stencil
// member), so the halo of a rank is every cell in {j} + stencil(j) for j in {i} + faces(i),
// i owned, that the rank does not own: up to three face rings deep. A two-stage step
// exchanges the halo twice (the state and the stage state); the time step is a minimum over
// the ranks. The paper runs one GPU (its multi-GPU work is left for the future); this file
// plans the exchange, and the caller moves the data.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <new>
#include <string>
#include <vector>

#include "gks_internal.h"

namespace {

uint64_t spread21(uint64_t v) {
  v &= 0x1fffffULL;
  v = (v | v << 32) & 0x1f00000000ffffULL;
  v = (v | v << 16) & 0x1f0000ff0000ffULL;
  v = (v | v << 8) & 0x100f00f00f00f00fULL;
  v = (v | v << 4) & 0x10c30c30c30c30c3ULL;
  v = (v | v << 2) & 0x1249249249249249ULL;
  return v;
}

}  // namespace

struct gks_partition {
  int nranks = 0, rank = 0;
  std::vector<int32_t> rank_of;          // caller cell -> owning rank
  std::vector<int64_t> owned;            // caller ids, Morton order
  std::vector<int64_t> halo;             // caller ids, by (owner rank, caller id)
  std::vector<int32_t> halo_owner;
  std::vector<std::vector<int64_t>> send;  // per peer rank: owned cells in its halo order
};

namespace {

// The halo of rank r: the cells outside r that the residuals of r's cells read, sorted by
// (owner rank, caller id).
void halo_of(const gks::HostMesh& h, const std::vector<int32_t>& rank_of, int r,
             std::vector<int64_t>& out) {
  const int64_t nc = h.n_cells;
  std::vector<char> mark(nc, 0);
  auto need_poly = [&](int32_t j) {  // internal id j: the cell itself and its big stencil
    const int32_t cj = h.perm[j];
    if (rank_of[cj] != r) mark[cj] = 1;
    for (int32_t k = h.st_ptr[j]; k < h.st_ptr[j + 1]; ++k) {
      const int32_t cm = h.perm[h.st_idx[k] & gks::kCellMask];
      if (rank_of[cm] != r) mark[cm] = 1;
    }
  };
  for (int64_t i = 0; i < nc; ++i) {
    if (rank_of[h.perm[i]] != r) continue;
    need_poly((int32_t)i);
    for (int32_t k = h.cf_ptr[i]; k < h.cf_ptr[i + 1]; ++k) {
      const int32_t e = h.cf_idx[k], f = e >> 1;
      const int32_t other = (e & 1) ? h.f_owner[f] : h.f_nb[f];
      if (other >= 0) need_poly(other);
    }
  }
  out.clear();
  for (int64_t c = 0; c < nc; ++c)
    if (mark[c]) out.push_back(c);
  std::stable_sort(out.begin(), out.end(),
                   [&](int64_t a, int64_t b) { return rank_of[a] < rank_of[b]; });
}

}  // namespace

extern "C" gks_status gks_partition_create(const gks_mesh* m, int nranks, int rank,
                                           gks_partition** out) {
  if (!out) return GKS_E_INVAL;
  *out = nullptr;
  if (!m || nranks < 1 || rank < 0 || rank >= nranks || nranks > m->h.n_cells) {
    gks::set_global_error("gks_partition_create: invalid argument");
    return GKS_E_INVAL;
  }
  const gks::HostMesh& h = m->h;
  const int64_t nc = h.n_cells;
  gks_partition* p = new (std::nothrow) gks_partition;
  if (!p) return GKS_E_NOMEM;
  try {
    p->nranks = nranks;
    p->rank = rank;
    // Morton order of the vertex means (ties by caller id)
    std::vector<std::pair<uint64_t, int32_t>> key(nc);
    for (int64_t i = 0; i < nc; ++i) {
      double x[3] = {0, 0, 0};
      for (int s = 0; s < 8; ++s)
        for (int a = 0; a < 3; ++a) x[a] += h.cell_x[(8 * i + s) * 3 + a] / 8.0;
      uint64_t k = 0;
      for (int a = 0; a < 3; ++a) {
        double u = (x[a] - h.lo[a]) / (h.hi[a] - h.lo[a]);
        u = std::min(std::max(u, 0.0), 1.0);
        k |= spread21((uint64_t)(u * 2097151.0)) << a;
      }
      key[i] = {k, h.perm[i]};
    }
    std::sort(key.begin(), key.end());
    // contiguous ranges: the first nc % nranks ranks take one cell more
    p->rank_of.assign(nc, 0);
    const int64_t base = nc / nranks, extra = nc % nranks;
    int64_t pos = 0;
    for (int q = 0; q < nranks; ++q) {
      const int64_t len = base + (q < extra ? 1 : 0);
      for (int64_t k = 0; k < len; ++k, ++pos) {
        p->rank_of[key[pos].second] = q;
        if (q == rank) p->owned.push_back(key[pos].second);
      }
    }
    halo_of(h, p->rank_of, rank, p->halo);
    p->halo_owner.resize(p->halo.size());
    for (size_t k = 0; k < p->halo.size(); ++k) p->halo_owner[k] = p->rank_of[p->halo[k]];
    // what each peer needs from this rank, in the peer's halo order
    p->send.assign(nranks, {});
    std::vector<int64_t> hq;
    for (int q = 0; q < nranks; ++q) {
      if (q == rank) continue;
      halo_of(h, p->rank_of, q, hq);
      for (int64_t c : hq)
        if (p->rank_of[c] == rank) p->send[q].push_back(c);
    }
  } catch (const std::bad_alloc&) {
    delete p;
    gks::set_global_error("gks_partition_create: host allocation failed");
    return GKS_E_NOMEM;
  }
  *out = p;
  return GKS_OK;
}

extern "C" gks_status gks_partition_counts(const gks_partition* p, int64_t* n_owned,
                                           int64_t* n_halo) {
  if (!p) return GKS_E_INVAL;
  if (n_owned) *n_owned = (int64_t)p->owned.size();
  if (n_halo) *n_halo = (int64_t)p->halo.size();
  return GKS_OK;
}

extern "C" gks_status gks_partition_cells(const gks_partition* p, int64_t* owned, int64_t* halo,
                                          int32_t* halo_owner) {
  if (!p) return GKS_E_INVAL;
  if (owned) std::copy(p->owned.begin(), p->owned.end(), owned);
  if (halo) std::copy(p->halo.begin(), p->halo.end(), halo);
  if (halo_owner) std::copy(p->halo_owner.begin(), p->halo_owner.end(), halo_owner);
  return GKS_OK;
}

extern "C" gks_status gks_partition_send(const gks_partition* p, int peer, int64_t* n,
                                         int64_t* cells) {
  if (!p || !n || peer < 0 || peer >= p->nranks) return GKS_E_INVAL;
  const std::vector<int64_t>& s = p->send[peer];
  *n = (int64_t)s.size();
  if (cells) std::copy(s.begin(), s.end(), cells);
  return GKS_OK;
}

extern "C" void gks_partition_destroy(gks_partition* p) { delete p; }

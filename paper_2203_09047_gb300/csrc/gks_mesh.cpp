// Host-side mesh ingest: face matching (with periodic images), reflecting walls, the big
// stencils and sub-stencils of Section 2, and the Morton reorder of cells and faces.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <tuple>
#include <vector>

#include "gks_internal.h"

namespace gks {
namespace {

// Paper vertex labels p1..pN -> degenerate-hexahedron slot (Section 2 relabelling).
const int kSlotTet[4] = {0, 1, 2, 4};
const int kSlotPyr[5] = {0, 1, 2, 3, 4};
const int kSlotPri[6] = {0, 1, 2, 4, 5, 6};
const int kSlotHex[8] = {0, 1, 2, 3, 4, 5, 6, 7};

struct FaceDef {
  int n;     // 3 or 4 vertices
  int v[4];  // 1-based paper labels
};
// Face labels F_1..F_P of Section 2 (prism F3 as {p1 p2 p5 p4}).
const FaceDef kFacesTet[4] = {{3, {1, 2, 3}}, {3, {1, 2, 4}}, {3, {2, 3, 4}}, {3, {3, 1, 4}}};
const FaceDef kFacesPyr[5] = {
    {3, {1, 2, 5}}, {3, {2, 3, 5}}, {3, {3, 4, 5}}, {3, {4, 1, 5}}, {4, {1, 2, 3, 4}}};
const FaceDef kFacesPri[5] = {
    {3, {1, 2, 3}}, {3, {4, 5, 6}}, {4, {1, 2, 5, 4}}, {4, {2, 3, 6, 5}}, {4, {3, 1, 4, 6}}};
const FaceDef kFacesHex[6] = {{4, {1, 2, 3, 4}}, {4, {1, 2, 6, 5}}, {4, {2, 3, 7, 6}},
                              {4, {3, 4, 8, 7}}, {4, {4, 1, 5, 8}}, {4, {5, 6, 7, 8}}};

int n_faces_of(int t) { return t == GKS_TET ? 4 : t == GKS_HEX ? 6 : 5; }
const FaceDef& face_def(int t, int p) {
  if (t == GKS_TET) return kFacesTet[p];
  if (t == GKS_PYR) return kFacesPyr[p];
  if (t == GKS_PRI) return kFacesPri[p];
  return kFacesHex[p];
}
int slot_of(int t, int label) {  // label 1-based
  if (t == GKS_TET) return kSlotTet[label - 1];
  if (t == GKS_PYR) return kSlotPyr[label - 1];
  if (t == GKS_PRI) return kSlotPri[label - 1];
  return kSlotHex[label - 1];
}

// Sub-stencils (Section 2): three local faces each; tetrahedra and pyramids add the other
// neighbours of one of those face neighbours (1-based local face, 0 = none).
struct SubRule {
  int8_t f[3];
  int8_t grow;
};
const SubRule kSubHex[8] = {{{1, 2, 3}, 0}, {{1, 3, 4}, 0}, {{1, 4, 5}, 0}, {{1, 5, 2}, 0},
                            {{6, 2, 3}, 0}, {{6, 3, 4}, 0}, {{6, 4, 5}, 0}, {{6, 5, 2}, 0}};
const SubRule kSubPri[6] = {{{1, 3, 4}, 0}, {{1, 4, 5}, 0}, {{1, 5, 3}, 0},
                            {{2, 3, 4}, 0}, {{2, 4, 5}, 0}, {{2, 5, 3}, 0}};
const SubRule kSubTet[4] = {{{1, 2, 3}, 1}, {{1, 2, 4}, 2}, {{2, 3, 4}, 3}, {{3, 1, 4}, 4}};
const SubRule kSubPyr[8] = {{{1, 2, 3}, 1}, {{2, 3, 4}, 2}, {{3, 4, 1}, 3}, {{4, 1, 2}, 4},
                            {{1, 2, 5}, 1}, {{2, 3, 5}, 2}, {{3, 4, 5}, 3}, {{4, 1, 5}, 4}};
int sub_rules(int t, const SubRule** r) {
  if (t == GKS_HEX) { *r = kSubHex; return 8; }
  if (t == GKS_PRI) { *r = kSubPri; return 6; }
  if (t == GKS_TET) { *r = kSubTet; return 4; }
  *r = kSubPyr;
  return 8;
}

Xf xf_compose(const Xf& a, const Xf& b) {  // a(b(x))
  Xf c;
  for (int k = 0; k < 3; ++k) {
    c.s[k] = (int8_t)(a.s[k] * b.s[k]);
    c.t[k] = a.s[k] * b.t[k] + a.t[k];
  }
  c.vflip = a.vflip ^ b.vflip;
  for (int k = 0; k < b.nw; ++k) c.w[c.nw++] = b.w[k];
  for (int k = 0; k < a.nw; ++k) {
    if (c.nw == 2) {
      c.nw = 3;  // more than two walls: rejected by the stencil builder
      break;
    }
    c.w[c.nw++] = a.w[k];
  }
  return c;
}
bool xf_equal(const Xf& a, const Xf& b, double tol) {
  for (int k = 0; k < 3; ++k)
    if (a.s[k] != b.s[k] || std::fabs(a.t[k] - b.t[k]) > tol) return false;
  return true;
}
bool xf_is_identity(const Xf& a, double tol) { return xf_equal(a, Xf(), tol); }

uint64_t spread21(uint64_t v) {  // interleave helper for a 63-bit Morton code
  v &= 0x1fffff;
  v = (v | v << 32) & 0x1f00000000ffffULL;
  v = (v | v << 16) & 0x1f0000ff0000ffULL;
  v = (v | v << 8) & 0x100f00f00f00f00fULL;
  v = (v | v << 4) & 0x10c30c30c30c30c3ULL;
  v = (v | v << 2) & 0x1249249249249249ULL;
  return v;
}

struct Nb {
  int32_t cell;  // caller id
  Xf xf;         // neighbour frame -> this cell's frame
};

}  // namespace

gks_status build_host_mesh(int64_t n_nodes, const double* xyz, int64_t n_cells,
                           const int8_t* cell_type, const int64_t* cell_nodes, const int bc[3],
                           const double lo[3], const double hi[3], int reorder, int min_stencil,
                           HostMesh& m, std::string& err) {
  if (n_nodes <= 0 || n_cells <= 0 || !xyz || !cell_type || !cell_nodes || !bc || !lo || !hi) {
    err = "empty mesh or null array";
    return GKS_E_INVAL;
  }
  if (reorder < GKS_REORDER_NONE || reorder > GKS_REORDER_RCM) {
    err = "unknown cell reorder";
    return GKS_E_INVAL;
  }
  if (min_stencil < 0 || min_stencil > kMaxStencil) {
    err = "min_stencil out of range";
    return GKS_E_INVAL;
  }
  if (n_cells >= (int64_t)kCellMask) {
    err = "too many cells";
    return GKS_E_INVAL;
  }
  double L[3], ext = 0;
  for (int a = 0; a < 3; ++a) {
    if (bc[a] != GKS_BC_PERIODIC && bc[a] != GKS_BC_REFLECT && bc[a] != GKS_BC_NOSLIP &&
        bc[a] != GKS_BC_FARFIELD) {
      err = "unknown boundary condition";
      return GKS_E_INVAL;
    }
    L[a] = hi[a] - lo[a];
    if (!(L[a] > 0)) {
      err = "empty bounding box";
      return GKS_E_INVAL;
    }
    ext = std::max(ext, L[a]);
    m.bc[a] = bc[a];
    m.lo[a] = lo[a];
    m.hi[a] = hi[a];
  }
  const double tol = 1e-9 * ext;
  const int64_t nc = n_cells;
  for (int64_t c = 0; c < nc; ++c) {
    const int t = cell_type[c];
    if (t != GKS_TET && t != GKS_PYR && t != GKS_PRI && t != GKS_HEX) {
      err = "cell " + std::to_string(c) + ": unknown type " + std::to_string(t);
      return GKS_E_INVAL;
    }
    for (int s = 0; s < 8; ++s) {
      const int64_t v = cell_nodes[8 * c + s];
      if (v < 0 || v >= n_nodes) {
        err = "cell " + std::to_string(c) + ": node index out of range";
        return GKS_E_INVAL;
      }
    }
  }

  // 1. one representative per set of periodic node images (sort by wrapped lattice key)
  std::vector<int64_t> rep(n_nodes);
  {
    const double q = 1e-7 * ext;
    std::vector<std::array<int64_t, 4>> keys(n_nodes);
    for (int64_t i = 0; i < n_nodes; ++i) {
      for (int a = 0; a < 3; ++a) {
        double x = xyz[3 * i + a];
        if (bc[a] == GKS_BC_PERIODIC && std::fabs(x - hi[a]) < tol) x = lo[a];
        keys[i][a] = (int64_t)std::llround((x - lo[a]) / q);
      }
      keys[i][3] = i;
    }
    std::sort(keys.begin(), keys.end());
    for (int64_t k = 0; k < n_nodes;) {
      int64_t e = k;
      int64_t first = keys[k][3];
      while (e < n_nodes && keys[e][0] == keys[k][0] && keys[e][1] == keys[k][1] &&
             keys[e][2] == keys[k][2]) {
        first = std::min(first, keys[e][3]);
        ++e;
      }
      for (int64_t j = k; j < e; ++j) rep[keys[j][3]] = first;
      k = e;
    }
  }

  // 2. match cell faces: sort (sorted representative ids, cell, local face)
  struct Rec {
    int64_t k[4];
    int32_t cell;
    int8_t lf;
  };
  std::vector<int32_t> fptr(nc + 1, 0);
  for (int64_t c = 0; c < nc; ++c) fptr[c + 1] = fptr[c] + n_faces_of(cell_type[c]);
  std::vector<Rec> recs(fptr[nc]);
  for (int64_t c = 0; c < nc; ++c) {
    const int t = cell_type[c];
    for (int p = 0; p < n_faces_of(t); ++p) {
      const FaceDef& fd = face_def(t, p);
      Rec r;
      for (int k = 0; k < 4; ++k)
        r.k[k] = k < fd.n ? rep[cell_nodes[8 * c + slot_of(t, fd.v[k])]] : -1;
      std::sort(r.k, r.k + fd.n);
      r.cell = (int32_t)c;
      r.lf = (int8_t)p;
      recs[fptr[c] + p] = r;
    }
  }
  std::sort(recs.begin(), recs.end(), [](const Rec& a, const Rec& b) {
    for (int k = 0; k < 4; ++k)
      if (a.k[k] != b.k[k]) return a.k[k] < b.k[k];
    if (a.cell != b.cell) return a.cell < b.cell;
    return a.lf < b.lf;
  });
  // neighbour table per (caller cell, local face) and the face list (caller ids for now)
  std::vector<Nb> nbs(fptr[nc]);
  struct FaceTmp {
    int32_t owner, nb;
    int8_t of, nf, wall;
    double shift[3];
  };
  std::vector<FaceTmp> faces;
  faces.reserve(recs.size() / 2 + 16);
  auto node_x = [&](int64_t id, int a) { return xyz[3 * id + a]; };
  for (size_t i = 0; i < recs.size();) {
    size_t e = i + 1;
    while (e < recs.size() && std::equal(recs[e].k, recs[e].k + 4, recs[i].k)) ++e;
    if (e - i > 2) {
      err = "a face is shared by more than two cells";
      return GKS_E_MESH;
    }
    FaceTmp f;
    f.owner = recs[i].cell;  // sorted: lower cell id (then lower local face) owns the face
    f.of = recs[i].lf;
    f.shift[0] = f.shift[1] = f.shift[2] = 0.0;
    const int to = cell_type[f.owner];
    const FaceDef& fo = face_def(to, f.of);
    if (e - i == 2) {
      f.nb = recs[i + 1].cell;
      f.nf = recs[i + 1].lf;
      f.wall = -1;
      const int tn = cell_type[f.nb];
      const FaceDef& fn = face_def(tn, f.nf);
      // translation from the neighbour's vertices to the owner's
      for (int k = 0; k < fo.n; ++k) {
        const int64_t vo = cell_nodes[8 * (int64_t)f.owner + slot_of(to, fo.v[k])];
        int64_t vn = -1;
        for (int j = 0; j < fn.n; ++j) {
          const int64_t w = cell_nodes[8 * (int64_t)f.nb + slot_of(tn, fn.v[j])];
          if (rep[w] == rep[vo]) vn = w;
        }
        for (int a = 0; a < 3; ++a) {
          const double d = node_x(vo, a) - node_x(vn, a);
          if (k == 0) {
            f.shift[a] = d;
          } else if (std::fabs(d - f.shift[a]) > 1e-6 * ext) {
            err = "periodic face vertices are not related by one translation";
            return GKS_E_MESH;
          }
        }
      }
      for (int a = 0; a < 3; ++a) {
        if (std::fabs(f.shift[a]) < tol) f.shift[a] = 0.0;
        else if (bc[a] != GKS_BC_PERIODIC) {
          err = "faces matched across a non-periodic axis";
          return GKS_E_MESH;
        }
      }
    } else {
      f.nb = -1;
      f.nf = -1;
      f.wall = -1;
      double plane = 0;
      for (int a = 0; a < 3 && f.wall < 0; ++a) {
        if (bc[a] == GKS_BC_PERIODIC) continue;
        for (int side = 0; side < 2 && f.wall < 0; ++side) {
          const double pl = side ? hi[a] : lo[a];
          bool on = true;
          for (int k = 0; k < fo.n; ++k)
            if (std::fabs(node_x(cell_nodes[8 * (int64_t)f.owner + slot_of(to, fo.v[k])], a) -
                          pl) > tol)
              on = false;
          if (on) {
            f.wall = (int8_t)(a + 3 * side + 6 * (bc[a] - GKS_BC_REFLECT));
            plane = pl;
          }
        }
      }
      if (f.wall < 0) {
        err = "cell " + std::to_string(f.owner) + " face " + std::to_string(f.of + 1) +
              ": unmatched face not on a reflecting boundary plane";
        return GKS_E_MESH;
      }
      f.shift[wall_axis(f.wall)] = 2.0 * plane;  // mirror: x' = -x + 2 plane on the wall axis
    }
    // neighbour table entries
    if (f.nb >= 0) {
      Nb a;
      a.cell = f.nb;
      for (int k = 0; k < 3; ++k) a.xf.t[k] = f.shift[k];
      nbs[fptr[f.owner] + f.of] = a;
      Nb b;
      b.cell = f.owner;
      for (int k = 0; k < 3; ++k) b.xf.t[k] = -f.shift[k];
      nbs[fptr[f.nb] + f.nf] = b;
    } else {
      Nb a;
      const int ax = wall_axis(f.wall);
      a.cell = f.owner;
      a.xf.s[ax] = -1;
      a.xf.t[ax] = f.shift[ax];
      a.xf.vflip = (uint8_t)(wall_farfield(f.wall) ? 0 : wall_noslip(f.wall) ? 7 : 1 << ax);
      a.xf.nw = 1;
      a.xf.w[0] = (int8_t)wall_plane(f.wall);
      nbs[fptr[f.owner] + f.of] = a;
    }
    faces.push_back(f);
    i = e;
  }

  // 3. cell order: by cell kind (so that 32-cell tiles hold cells with (nearly) the same
  //    stencil sizes), then the Morton order of the vertex mean (default), the reverse
  //    Cuthill-McKee order of the face graph, or the caller's order
  std::vector<int32_t> perm(nc), inv(nc);
  {
    std::vector<uint64_t> key(nc);
    if (reorder == GKS_REORDER_MORTON) {
      for (int64_t c = 0; c < nc; ++c) {
        double x[3] = {0, 0, 0};
        for (int s = 0; s < 8; ++s)
          for (int a = 0; a < 3; ++a) x[a] += node_x(cell_nodes[8 * c + s], a) / 8.0;
        uint64_t k = 0;
        for (int a = 0; a < 3; ++a) {
          double u = (x[a] - lo[a]) / L[a];
          u = std::min(std::max(u, 0.0), 1.0);
          k |= spread21((uint64_t)(u * 2097151.0)) << a;
        }
        key[c] = k;
      }
    } else if (reorder == GKS_REORDER_RCM) {
      // Cuthill-McKee: breadth-first from an unvisited cell of least degree, neighbours in
      // increasing degree (ties by id); the reverse of the visit order is the key
      auto degree = [&](int64_t c) {
        int d = 0;
        for (int p = 0; p < n_faces_of(cell_type[c]); ++p)
          if (nbs[fptr[c] + p].xf.nw == 0) ++d;
        return d;
      };
      std::vector<int32_t> by_deg(nc);
      std::iota(by_deg.begin(), by_deg.end(), 0);
      std::stable_sort(by_deg.begin(), by_deg.end(),
                       [&](int32_t a, int32_t b) { return degree(a) < degree(b); });
      std::vector<char> seen(nc, 0);
      std::vector<int32_t> order;
      order.reserve(nc);
      std::vector<int32_t> next;
      for (int32_t s : by_deg) {
        if (seen[s]) continue;
        seen[s] = 1;
        size_t head = order.size();
        order.push_back(s);
        while (head < order.size()) {
          const int32_t c = order[head++];
          next.clear();
          for (int p = 0; p < n_faces_of(cell_type[c]); ++p) {
            const Nb& b = nbs[fptr[c] + p];
            if (b.xf.nw == 0 && !seen[b.cell]) {
              seen[b.cell] = 1;
              next.push_back(b.cell);
            }
          }
          std::stable_sort(next.begin(), next.end(), [&](int32_t a, int32_t b) {
            const int da = degree(a), db = degree(b);
            return da != db ? da < db : a < b;
          });
          order.insert(order.end(), next.begin(), next.end());
        }
      }
      for (int64_t i = 0; i < nc; ++i) key[order[i]] = (uint64_t)(nc - 1 - i);
    } else {
      for (int64_t c = 0; c < nc; ++c) key[c] = (uint64_t)c;
    }
    std::vector<std::tuple<int, uint64_t, int32_t>> code(nc);
    for (int64_t c = 0; c < nc; ++c) code[c] = std::make_tuple((int)cell_type[c], key[c], (int32_t)c);
    std::sort(code.begin(), code.end());
    for (int64_t i = 0; i < nc; ++i) {
      perm[i] = std::get<2>(code[i]);
      inv[perm[i]] = (int32_t)i;
    }
  }

  // 4. faces: oriented vertex lists, then sorted by (internal owner, internal neighbour)
  std::vector<int32_t> forder(faces.size());
  std::iota(forder.begin(), forder.end(), 0);
  std::sort(forder.begin(), forder.end(), [&](int32_t a, int32_t b) {
    const int32_t oa = inv[faces[a].owner], ob = inv[faces[b].owner];
    if (oa != ob) return oa < ob;
    const int32_t na = faces[a].nb >= 0 ? inv[faces[a].nb] : -1;
    const int32_t nbb = faces[b].nb >= 0 ? inv[faces[b].nb] : -1;
    if (na != nbb) return na < nbb;
    return faces[a].of < faces[b].of;
  });
  const int64_t nf = (int64_t)faces.size();
  m.n_cells = nc;
  m.n_faces = nf;
  m.perm = perm;
  m.f_owner.resize(nf);
  m.f_nb.resize(nf);
  m.f_wall.resize(nf);
  m.f_vert.resize(12 * nf);
  m.f_shift.resize(3 * nf);
  std::vector<int32_t> face_new(nf);
  for (int64_t k = 0; k < nf; ++k) face_new[forder[k]] = (int32_t)k;
  for (int64_t k = 0; k < nf; ++k) {
    const FaceTmp& f = faces[forder[k]];
    m.f_owner[k] = inv[f.owner];
    m.f_nb[k] = f.nb >= 0 ? inv[f.nb] : -1;
    m.f_wall[k] = f.wall;
    for (int a = 0; a < 3; ++a) m.f_shift[3 * k + a] = f.nb >= 0 ? f.shift[a] : 0.0;
    // owner-side vertex list, oriented out of the owner, smallest node id first
    const int to = cell_type[f.owner];
    const FaceDef& fd = face_def(to, f.of);
    int64_t ids[4];
    for (int j = 0; j < fd.n; ++j) ids[j] = cell_nodes[8 * (int64_t)f.owner + slot_of(to, fd.v[j])];
    double cm[3] = {0, 0, 0};
    for (int s = 0; s < 8; ++s)
      for (int a = 0; a < 3; ++a) cm[a] += node_x(cell_nodes[8 * (int64_t)f.owner + s], a) / 8.0;
    auto vx = [&](int j, int a) { return node_x(ids[std::min(j, fd.n - 1)], a); };
    // X_eta x X_zeta at the face centre for the slot layout (-,-) (-,+) (+,+) (+,-)
    double xe[3], xz[3], ctr[3];
    for (int a = 0; a < 3; ++a) {
      xe[a] = 0.5 * (-vx(0, a) - vx(1, a) + vx(2, a) + vx(3, a));
      xz[a] = 0.5 * (-vx(0, a) + vx(1, a) + vx(2, a) - vx(3, a));
      ctr[a] = 0.25 * (vx(0, a) + vx(1, a) + vx(2, a) + vx(3, a));
    }
    const double nrm[3] = {xe[1] * xz[2] - xe[2] * xz[1], xe[2] * xz[0] - xe[0] * xz[2],
                           xe[0] * xz[1] - xe[1] * xz[0]};
    double dot = 0;
    for (int a = 0; a < 3; ++a) dot += nrm[a] * (ctr[a] - cm[a]);
    if (dot < 0) std::reverse(ids, ids + fd.n);
    int first = 0;
    for (int j = 1; j < fd.n; ++j)
      if (ids[j] < ids[first]) first = j;
    std::rotate(ids, ids + first, ids + fd.n);
    for (int j = 0; j < 4; ++j)
      for (int a = 0; a < 3; ++a) m.f_vert[12 * k + 3 * j + a] = node_x(ids[std::min(j, fd.n - 1)], a);
  }

  // 5. cells in internal order: slot coordinates and face incidences
  m.type.resize(nc);
  m.cell_x.resize(24 * nc);
  m.cf_ptr.assign(nc + 1, 0);
  for (int64_t i = 0; i < nc; ++i) {
    const int32_t c = perm[i];
    m.type[i] = cell_type[c];
    for (int s = 0; s < 8; ++s)
      for (int a = 0; a < 3; ++a) m.cell_x[24 * i + 3 * s + a] = node_x(cell_nodes[8 * (int64_t)c + s], a);
    m.cf_ptr[i + 1] = m.cf_ptr[i] + n_faces_of(cell_type[c]);
  }
  // face id per (caller cell, local face)
  std::vector<int32_t> lf_face(fptr[nc], -1);
  for (int64_t k = 0; k < nf; ++k) {
    const FaceTmp& f = faces[forder[k]];
    lf_face[fptr[f.owner] + f.of] = (int32_t)k << 1;
    if (f.nb >= 0) lf_face[fptr[f.nb] + f.nf] = ((int32_t)k << 1) | 1;
  }
  m.cf_idx.resize(m.cf_ptr[nc]);
  for (int64_t i = 0; i < nc; ++i) {
    const int32_t c = perm[i];
    for (int p = 0; p < n_faces_of(cell_type[c]); ++p) m.cf_idx[m.cf_ptr[i] + p] = lf_face[fptr[c] + p];
  }

  // 6. stencils (Section 2) per internal cell
  m.st_ptr.assign(nc + 1, 0);
  m.n_sub.resize(nc);
  m.sb_ptr.assign(nc + 1, 0);
  m.sub_cnt.assign(nc, 0);
  m.st_idx.clear();
  m.st_walls.clear();
  m.st_xf.clear();
  m.st_sub.clear();
  std::vector<Nb> list;
  for (int64_t i = 0; i < nc; ++i) {
    const int32_t c = perm[i];
    const int t = cell_type[c];
    const int P = n_faces_of(t);
    list.clear();
    auto find_or_add = [&](const Nb& e) -> int {
      if (e.cell == c && xf_is_identity(e.xf, tol)) return -1;
      for (size_t k = 0; k < list.size(); ++k)
        if (list[k].cell == e.cell && xf_equal(list[k].xf, e.xf, tol)) return (int)k;
      list.push_back(e);
      return (int)list.size() - 1;
    };
    auto ring2 = [&](int p, std::vector<Nb>& out) {  // neighbours of the neighbour across p
      const Nb& n1 = nbs[fptr[c] + p];
      const int tn = cell_type[n1.cell];
      for (int q = 0; q < n_faces_of(tn); ++q) {
        const Nb& n2 = nbs[fptr[n1.cell] + q];
        Nb e;
        e.cell = n2.cell;
        e.xf = xf_compose(n1.xf, n2.xf);
        out.push_back(e);
      }
    };
    for (int p = 0; p < P; ++p) find_or_add(nbs[fptr[c] + p]);
    std::vector<Nb> r2;
    for (int p = 0; p < P; ++p) {
      r2.clear();
      ring2(p, r2);
      for (const Nb& e : r2) find_or_add(e);
    }
    // optional third ring (a reading, not in the paper): a big stencil with fewer than
    // min_stencil members takes the face neighbours of its members, member by member in
    // stencil order and face by face in face-label order, until it has min_stencil members;
    // images that cross more than two wall planes are skipped
    if ((int)list.size() < min_stencil) {
      const size_t n2 = list.size();
      for (size_t k = 0; k < n2 && (int)list.size() < min_stencil; ++k) {
        const Nb mk = list[k];
        const int tk = cell_type[mk.cell];
        for (int q = 0; q < n_faces_of(tk) && (int)list.size() < min_stencil; ++q) {
          Nb e;
          e.cell = nbs[fptr[mk.cell] + q].cell;
          e.xf = xf_compose(mk.xf, nbs[fptr[mk.cell] + q].xf);
          if (e.xf.nw > 2) continue;
          find_or_add(e);
        }
      }
    }
    const SubRule* rules;
    const int M = sub_rules(t, &rules);
    std::vector<uint8_t> sub(list.size(), 0);
    for (int s = 0; s < M; ++s) {
      std::vector<int> members;
      auto put = [&](const Nb& e) {
        const int k = find_or_add(e);
        if (k < 0) return;
        if (std::find(members.begin(), members.end(), k) == members.end()) members.push_back(k);
      };
      for (int j = 0; j < 3; ++j) put(nbs[fptr[c] + rules[s].f[j] - 1]);
      if (rules[s].grow) {
        r2.clear();
        ring2(rules[s].grow - 1, r2);
        for (const Nb& e : r2) put(e);
      }
      sub.resize(list.size(), 0);
      for (int k : members) sub[k] |= (uint8_t)(1u << s);
    }
    if ((int)list.size() > kMaxStencil) {
      err = "cell " + std::to_string(c) + ": stencil larger than " + std::to_string(kMaxStencil);
      return GKS_E_MESH;
    }
    m.n_sub[i] = (int8_t)M;
    int pairs = 0;
    for (size_t k = 0; k < list.size(); ++k) {
      const Nb& e = list[k];
      if (e.xf.nw > 2) {
        err = "cell " + std::to_string(c) + ": a stencil member crosses more than two walls";
        return GKS_E_MESH;
      }
      m.st_idx.push_back(inv[e.cell] | ((int32_t)e.xf.vflip << kFlipShift));
      m.st_walls.push_back((uint8_t)((e.xf.nw > 0 ? e.xf.w[0] + 1 : 0) |
                                     (e.xf.nw > 1 ? (e.xf.w[1] + 1) << 3 : 0)));
      for (int a = 0; a < 3; ++a) m.st_xf.push_back((double)e.xf.s[a]);
      for (int a = 0; a < 3; ++a) m.st_xf.push_back(e.xf.t[a]);
      m.st_sub.push_back(sub[k]);
      pairs += __builtin_popcount(sub[k]);
    }
    m.st_ptr[i + 1] = m.st_ptr[i] + (int32_t)list.size();
    m.sb_ptr[i + 1] = m.sb_ptr[i] + pairs;
    uint64_t cnt = 0;  // members per sub-stencil, one byte each
    for (int s = 0; s < M; ++s) {
      uint64_t c = 0;
      for (size_t k = 0; k < list.size(); ++k) c += (sub[k] >> s) & 1u;
      cnt |= c << (8 * s);
    }
    m.sub_cnt[i] = cnt;
  }
  // 7. 32-cell tiles: stencil entries interleaved across the tile's lanes, padded to the tile's
  //    largest stencil (padding points at the cell itself, whose difference is zero) and the
  //    tile's largest member count per sub-stencil
  const int64_t nt = (nc + kTile - 1) / kTile;
  m.n_tiles = nt;
  m.t_K.assign(nt, 0);
  m.t_cnt.assign(nt, 0);
  m.t_st.assign(nt + 1, 0);
  m.t_sb.assign(nt + 1, 0);
  for (int64_t t = 0; t < nt; ++t) {
    int K = 0;
    int cmax[kMaxSub] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t c = t * kTile; c < std::min<int64_t>(nc, (t + 1) * kTile); ++c) {
      K = std::max(K, m.st_ptr[c + 1] - m.st_ptr[c]);
      for (int q = 0; q < kMaxSub; ++q) cmax[q] = std::max(cmax[q], (int)((m.sub_cnt[c] >> (8 * q)) & 0xff));
    }
    uint64_t cw = 0;
    int tot = 0;
    for (int q = 0; q < kMaxSub; ++q) {
      cw |= (uint64_t)cmax[q] << (8 * q);
      tot += cmax[q];
    }
    m.t_K[t] = K;
    m.t_cnt[t] = cw;
    m.t_st[t + 1] = m.t_st[t] + K;
    m.t_sb[t + 1] = m.t_sb[t] + tot;
  }
  m.t_idx.assign((size_t)m.t_st[nt] * kTile, 0);
  for (int64_t t = 0; t < nt; ++t)
    for (int l = 0; l < kTile; ++l) {
      const int64_t c = t * kTile + l;
      const int Kc = c < nc ? m.st_ptr[c + 1] - m.st_ptr[c] : 0;
      for (int k = 0; k < m.t_K[t]; ++k)
        m.t_idx[((size_t)m.t_st[t] + k) * kTile + l] =
            k < Kc ? m.st_idx[m.st_ptr[c] + k] : (int32_t)(c < nc ? c : t * kTile);
    }
  // 8. reverse stencil (counting sort by referenced cell, positions in increasing order)
  m.rs_ptr.assign(nc + 1, 0);
  for (int64_t t = 0; t < nt; ++t)
    for (int l = 0; l < kTile; ++l) {
      const int64_t c = t * kTile + l;
      if (c >= nc) continue;
      for (int k = 0; k < m.st_ptr[c + 1] - m.st_ptr[c]; ++k)
        ++m.rs_ptr[(m.t_idx[((size_t)m.t_st[t] + k) * kTile + l] & kCellMask) + 1];
    }
  for (int64_t c = 0; c < nc; ++c) m.rs_ptr[c + 1] += m.rs_ptr[c];
  m.rs_pos.assign(m.rs_ptr[nc], 0);
  {
    std::vector<int32_t> fill(m.rs_ptr.begin(), m.rs_ptr.end() - 1);
    for (int64_t t = 0; t < nt; ++t)
      for (int k = 0; k < m.t_K[t]; ++k)
        for (int l = 0; l < kTile; ++l) {
          const int64_t c = t * kTile + l;
          if (c >= nc || k >= m.st_ptr[c + 1] - m.st_ptr[c]) continue;
          const size_t pos = ((size_t)m.t_st[t] + k) * kTile + l;
          m.rs_pos[fill[m.t_idx[pos] & kCellMask]++] = (int32_t)pos;
        }
  }
  return GKS_OK;
}

}  // namespace gks

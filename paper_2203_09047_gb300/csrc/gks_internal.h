// Internal data structures shared by the host mesh builder, the device precompute and the
// hot-path kernels of the GB300 gas-kinetic solver.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/gks.h"

namespace gks {

// Stencil entries carry the cell index in the low bits and a 3-bit mask of mirrored axes
// (momentum components that change sign) in the top bits.
constexpr int kFlipShift = 28;
constexpr int32_t kCellMask = (1 << kFlipShift) - 1;
constexpr int kMaxStencil = 64;  // largest big stencil accepted
constexpr int kMaxSub = 8;       // largest number of sub-stencils (hexahedra, pyramids)
constexpr int kTile = 32;        // cells per tile of the interleaved stencil layouts

// Affine per-axis map x' = s x + t between cell frames (periodic shift or mirror image), with
// the wall planes (axis + 3 side) the image was reflected across, in the order they apply, and
// the momentum components that end up negated (vflip bit j). A stencil member crosses at most
// two walls (a face of the cell and a face of a neighbour).
struct Xf {
  int8_t s[3] = {1, 1, 1};
  double t[3] = {0, 0, 0};
  uint8_t vflip = 0;
  int8_t nw = 0;
  int8_t w[2] = {-1, -1};
};
// Wall code of a face: -1 interior; axis + 3 side for a slip wall, 6 + axis + 3 side for a
// no-slip wall, 12 + axis + 3 side for a far-field plane.
inline int wall_axis(int code) { return code % 3; }
inline int wall_plane(int code) { return code % 6; }
inline bool wall_noslip(int code) { return code >= 6 && code < 12; }
inline bool wall_farfield(int code) { return code >= 12; }
// Values per boundary plane in the device plane table: wall velocity (3), wall temperature,
// far-field state (5), padding.
constexpr int kPlaneStride = 12;

// Host-side mesh after topology, stencil and ordering work. Cells and faces are in the
// internal (Morton) order; perm maps internal cell -> caller cell.
struct HostMesh {
  int64_t n_cells = 0, n_faces = 0;
  int bc[3] = {0, 0, 0};
  double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  std::vector<int32_t> perm;           // internal -> caller
  std::vector<int8_t> type;            // internal order
  std::vector<double> cell_x;          // [n][8][3] slot coordinates (internal order)
  // faces
  std::vector<int32_t> f_owner, f_nb;  // internal cell ids; nb = -1 on a reflecting wall
  std::vector<int8_t> f_wall;          // wall code (see wall_plane) or -1
  std::vector<double> f_vert;          // [nf][4][3] oriented vertices in the owner frame
  std::vector<double> f_shift;         // [nf][3] neighbour frame -> owner frame translation
  // cell -> face incidence, fixed local-face order: (face << 1) | (1 if the cell is the nb side)
  std::vector<int32_t> cf_ptr, cf_idx;
  // big stencil (without the cell itself) and sub-stencil membership
  std::vector<int32_t> st_ptr, st_idx;  // st_idx: cell | flip mask << kFlipShift
  std::vector<double> st_xf;            // [n_st][6]: s[3], t[3] of the member transform
  std::vector<uint8_t> st_walls;        // wall planes crossed: (w0 + 1) | (w1 + 1) << 3, 0 none
  std::vector<uint8_t> st_sub;          // bit m set if the member is in sub-stencil m
  std::vector<int8_t> n_sub;            // M per cell
  std::vector<int32_t> sb_ptr;          // offset of each cell's (member, sub-stencil) pairs
  std::vector<uint64_t> sub_cnt;        // byte s: number of members of sub-stencil s
  // 32-cell tiles (cells 32 t .. 32 t + 31)
  int64_t n_tiles = 0;
  std::vector<int32_t> t_K;             // largest stencil of the tile
  std::vector<uint64_t> t_cnt;          // byte s: largest member count of sub-stencil s
  std::vector<int32_t> t_st, t_sb;      // prefix sums of t_K and of the t_cnt bytes
  std::vector<int32_t> t_idx;           // [t_st[nt]][32] interleaved stencil entries
  // reverse stencil: for each cell, the tile-layout positions (t_st[t] + k) 32 + lane of the
  // stencil entries that reference it (real entries only), in increasing position
  std::vector<int32_t> rs_ptr, rs_pos;
};

struct DeviceGeom;  // defined in the CUDA sources

}  // namespace gks

struct gks_mesh {
  gks::HostMesh h;
};

namespace gks {
// Set the text returned by gks_last_error(NULL) / gks_mesh_last_error() on this thread.
void set_global_error(const char* msg);
// Host mesh construction (gks_mesh.cpp). Returns a status and fills err.
gks_status build_host_mesh(int64_t n_nodes, const double* xyz, int64_t n_cells,
                           const int8_t* cell_type, const int64_t* cell_nodes, const int bc[3],
                           const double lo[3], const double hi[3], int reorder, int min_stencil,
                           HostMesh& m,
                           std::string& err);
}  // namespace gks

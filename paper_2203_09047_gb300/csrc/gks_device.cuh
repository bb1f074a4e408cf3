// Device-side declarations shared by the CUDA translation units: the device copy of the mesh,
// the precomputed geometry, and the kernel launchers.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "gks_internal.h"

namespace gks {

// Storage layouts of the hot path.
//  - gather copy of the state, 48 bytes per cell: FP32 path [hi0..hi4, lo0..lo4, 0, 0] with
//    hi = (float)q and lo = (float)(q - hi); FP64 path [q0..q4, 0];
//  - tiles of 32 consecutive cells; within a tile every per-member array is interleaved over the
//    32 lanes: stencil entries [t_st[t] + k][32], pseudo-inverse rows [(t_st[t] + k) 9 + n][32],
//    sub-stencil entries {B_0, B_1, B_2, member index} [(t_sb[t] + slot) 4 + c][32], padded to
//    the tile's largest stencil and per-sub-stencil counts (padding contributes zero);
//  - cell polynomials: kPolyStride values per cell, variable v at offset 10 v;
//  - face fluxes: kFaceStride values per face (F^n 0..4, dF/dt 5..9).
template <class R>
struct Lay;
template <>
struct Lay<float> {
  static constexpr int apad = 12, gq = 12;
};
template <>
struct Lay<double> {
  static constexpr int apad = 10, gq = 6;
};
constexpr int kPolyStride = 52;
constexpr int kFaceStride = 12;

// Error bits of the device status word.
enum : int {
  kErrInverted = 1,     // a cell Jacobian <= 0 at a quadrature point
  kErrSingular = 2,     // a least-squares system is rank deficient
  kErrNonphysical = 4,  // rho <= 0, p <= 0 or NaN
  kErrBigStencil = 8,
  kErrTimeout = 16      // a bounded wait on an asynchronous copy ran out
};

// Contiguous ranges of tiles whose first cell has the same kind (cells are ordered by kind
// first, so there is one range per kind present). Each range records its largest stencil K, its
// largest sum S of per-sub-stencil member counts and its largest number M of sub-stencil slots;
// the reconstruction is launched once per range with shared memory sized for that range.
constexpr int kMaxTileRanges = 8;
struct TileRanges {
  int n = 0;
  int64_t t0[kMaxTileRanges] = {}, t1[kMaxTileRanges] = {};
  int K[kMaxTileRanges] = {}, S[kMaxTileRanges] = {}, M[kMaxTileRanges] = {};
  // uniform ranges: every tile has the first tile's stencil size and sub-stencil counts, so
  // the tile's offsets into the interleaved arrays follow from its index
  int uni[kMaxTileRanges] = {};
  uint64_t cnt[kMaxTileRanges] = {};
  int64_t st0[kMaxTileRanges] = {}, sb0[kMaxTileRanges] = {};
};

// Mesh arrays on the device (internal order).
struct DevMesh {
  int64_t nc = 0, nf = 0, nst = 0, nsb = 0;
  int kmax = 0;  // largest big stencil
  int32_t* perm = nullptr;
  int8_t* type = nullptr;
  double* cell_x = nullptr;   // [nc][24]
  int32_t* f_owner = nullptr;
  int32_t* f_nb = nullptr;
  int8_t* f_wall = nullptr;
  double* f_vert = nullptr;   // [nf][12]
  double* f_shift = nullptr;  // [nf][3]
  int32_t* cf_ptr = nullptr;
  int32_t* cf_idx = nullptr;
  int64_t ncf = 0;  // cell-face entries
  int32_t* st_ptr = nullptr;
  int32_t* st_idx = nullptr;
  double* st_xf = nullptr;    // [nst][6]
  uint8_t* st_sub = nullptr;
  int8_t* n_sub = nullptr;
  int32_t* sb_ptr = nullptr;
  uint64_t* sub_cnt = nullptr;
  int64_t n_tiles = 0, n_tslots = 0, n_tsb = 0;
  int32_t* t_K = nullptr;
  uint64_t* t_cnt = nullptr;
  int32_t* t_st = nullptr;
  int32_t* t_sb = nullptr;
  int32_t* t_idx = nullptr;
  TileRanges rr;
  // ghost cells of moving no-slip walls: stencil entries whose image's flow variables are not a
  // sign change of the source cell's (Section 2: ghost variables from the boundary condition)
  // point at slot nc + g of the gather copies, refreshed before each reconstruction from cell
  // g_src[g] by the linear map g_map[g] = (s[3], a[3], b, c[3]):
  //   rho -> rho, m_j -> s_j m_j + a_j rho, E -> E + b rho + c . m
  // (g_mapf: the same ten values as float-float pairs for the FP32 path).
  int64_t ng = 0;
  int32_t* g_src = nullptr;
  double* g_map = nullptr;
  float* g_mapf = nullptr;
  // slots whose image crossed a far-field plane are not linear: g_chain holds their planes
  // ((w0 + 1) | (w1 + 1) << 3, applied in order, 0 for a linear slot) and bcs the box condition
  // of each axis (2 bits per axis)
  uint8_t* g_chain = nullptr;
  int bcs = 0;
  // boundary planes (axis + 3 side): wall velocity and temperature, far-field state,
  // [6][kPlaneStride] in FP64 and FP32 (see WallData)
  double* wall64 = nullptr;
  float* wall32 = nullptr;
};
template <class R>
inline const R* wall_table(const DevMesh& m);
template <>
inline const double* wall_table<double>(const DevMesh& m) { return m.wall64; }
template <>
inline const float* wall_table<float>(const DevMesh& m) { return m.wall32; }

// FP64 geometry (always kept).
struct Geo64 {
  double* vol = nullptr;     // [nc]
  double* ivol = nullptr;    // [nc] 1 / |Omega|
  double* cen = nullptr;     // [nc][3]
  double* h = nullptr;       // [nc] |Omega|^(1/3)
  double* mom = nullptr;     // [6][nc] second central moments / (|Omega| h^2): xx yy zz xy xz yz
  double* hdt = nullptr;     // [nc] |Omega| / largest face area
  double* farea = nullptr;   // [nf]
};

// Geometry in the arithmetic precision R of the hot path.
template <class R>
struct GeoR {
  R* Ap = nullptr;   // pseudo-inverse rows, tile-interleaved
  R* Bp = nullptr;   // sub-stencil entries [slot][lane][4] (3 coefficients, member index)
  R* mom = nullptr;  // [6][nc]
  R* h = nullptr;    // [nc]
  R* fgp = nullptr;  // [10][4 nf]: dl(3) dr(3) n1(3) w, index 4 f + gauss point
  R* ivol = nullptr; // 1/|Omega|: [nc] (FP64 path) or [nc][2] float-float pairs (FP32 path)
};

// Parameters of the hot kernels.
template <class R>
struct KParams {
  R gamma, K, mu, tau_eps, tau_C, pr_fix;
  int flux_mode, tau_model;
  R weno_gamma, weno_eps;
  int weno_pow;
  R T_ref, mu_pow;  // power-law viscosity (the boundary planes live in DevMesh::wall64/wall32)
  int gp_fallback;  // first-order state at Gauss points whose reconstruction is non-physical
  // test hook (gks_debug_recon_wait): bounded-wait limit of the reconstruction's bulk copies
  // (0: the default) and whether the copies are withheld
  int wait_tries = 0;
  int withhold = 0;
};

// ---- precompute (gks_geom.cu) -------------------------------------------------------------
void launch_geom_cells(const DevMesh& m, const Geo64& g, int* flag, cudaStream_t st);
template <class R>
void launch_geom_faces(const DevMesh& m, const Geo64& g, GeoR<R>& gr, cudaStream_t st);
void launch_geom_hdt(const DevMesh& m, const Geo64& g, cudaStream_t st);
template <class R>
void launch_geom_ls(const DevMesh& m, const Geo64& g, GeoR<R>& gr, int* flag, int* bad_cell,
                    cudaStream_t st);
template <class R>
void launch_cast_cells(const DevMesh& m, const Geo64& g, GeoR<R>& gr, cudaStream_t st);
void launch_cell_quadrature(const DevMesh& m, double* xq, double* wq, cudaStream_t st);
// Unit normal out of the owner and area of every face, [nf][4] in precision R.
template <class R>
void launch_face_normals(const DevMesh& m, R* out, cudaStream_t st);

// ---- hot path (gks_hot.cu) ----------------------------------------------------------------
// Auxiliary streams on which the reconstruction's tile ranges run concurrently with the first
// one (forked from and joined back into the solver's stream with events).
struct ForkJoin {
  int n = 0;  // auxiliary streams available
  cudaStream_t aux[kMaxTileRanges - 1] = {};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[kMaxTileRanges - 1] = {};
};
// fj == nullptr: the ranges run one after the other on st.
template <class R>
void launch_recon(const DevMesh& m, const GeoR<R>& g, const KParams<R>& p, const R* QA,
                  R* poly, int* flag, cudaStream_t st, const ForkJoin* fj = nullptr);
template <class R>
void launch_flux(const DevMesh& m, const GeoR<R>& g, const KParams<R>& p, const R* poly,
                 const R* QA, double dt, R* fface, int* flag, cudaStream_t st);
// Residual output: L = -(1/|Omega|) sum_f s_f F_f and Lt likewise from dF/dt, in FP64.
template <class R>
void launch_gather(const DevMesh& m, const Geo64& g, const R* fface, double* L, double* Lt,
                   cudaStream_t st);
// Two-stage combinations on caller arrays (gks_s2o4_stage, gks_s2o4_stage_vjp).
void launch_s2o4_stage(int64_t n, int stage, double dt, const double* Q, const double* L,
                       const double* Lt, const double* Lts, double* out, cudaStream_t st);
void launch_s2o4_stage_vjp(int64_t n, int stage, double dt, const double* g, double* gQ,
                           double* gL, double* gLt, double* gLts, cudaStream_t st);
// One stage of the fourth-order update on the gather copy QA, which holds the state:
// stage 1 stores L, Lt (FP64 values, or float-float pairs in the same 8 bytes on the FP32 path)
// and writes Q* to QsA; stage 2 reads them and writes Q^{n+1} to QA.
// Q64 != nullptr (FP32 path only): FP64 face sums and update of the FP64 master state Q64
// [5][nc] with the FP64 inverse volumes ivol64, L and Lt in FP64.
template <class R>
void launch_stage(const DevMesh& m, const GeoR<R>& g, const R* fface, int stage, double dt,
                  void* L, void* Lt, R* QA, R* QsA, int* flag, cudaStream_t st,
                  double* Q64 = nullptr, const double* ivol64 = nullptr);
// Implicit step (Section 4) on the gather copy QA (the state), after the reconstruction and
// flux of Q^n: jacobi_init forms |Omega| Res = s + dt/2 st from the face sums, the diagonal
// D = |Omega|/dt + 1/2 sum_f r_f S_f, the per-entry factors hrs = 1/2 r_f S_f (cell-face CSR
// order) and dQ0 = |Omega| Res / D; each jacobi_sweep forms dQ^(k) from dQ^(k-1), the last one
// (last != 0) writes Q^n + dQ to QAout (the other gather copy) in place of dQ. Buffers are in precision R: Rv, dQ
// [5][nc], D [nc], hrs [cf entries]; fn is [nf][4] from launch_face_normals.
template <class R>
void launch_jacobi_init(const DevMesh& m, const R* fface, const R* fn, const double* vol,
                        double dt, const R* QA, R* Rv, R* D, R* hrs, R* dQ0, const KParams<R>& kp,
                        cudaStream_t st);
template <class R>
void launch_jacobi_sweep(const DevMesh& m, const R* fn, const R* QA, const R* Rv, const R* D,
                         const R* hrs, const R* dQin, R* dQout, int last, R* QAout,
                         const KParams<R>& kp, int* flag, cudaStream_t st);

// The state [5][nc] in FP64 (internal order) from its gather copy.
template <class R>
void launch_unpack(int64_t nc, const R* QA, double* Q, cudaStream_t st);
template <class R>
void launch_permute_in(int64_t nc, const int32_t* perm, const double* src, double* dst, R* gq,
                       cudaStream_t st);
void launch_permute_out(int64_t nc, const int32_t* perm, const double* src, double* dst,
                        cudaStream_t st);
void launch_check_state(int64_t nc, const double* Q, double gamma, int* flag, cudaStream_t st);
void launch_dt(int64_t nc, const double* Q, const double* hdt, double gamma, double mu, int power,
               double T_ref, double mu_pow, double* partial, int nblocks, double* out,
               cudaStream_t st);
int dt_blocks(int64_t nc);

// ---- adjoint (gks_adjoint.cu) --------------------------------------------------------------
// gQ = (dL/dQ)^T gL + (dLt/dQ)^T gLt on internal-order arrays; poly holds the forward
// reconstruction of the state whose FP64 gather copy is QA.
void launch_vjp(const DevMesh& m, const Geo64& g64, const GeoR<double>& g, const KParams<double>& p,
                const double* QA, const double* poly, const double* gL, const double* gLt,
                double dt, double* gpf, double* gpc, double* gdq, double* gq0, double* gQ,
                const int32_t* rs_ptr, const int32_t* rs_pos, int* flag, cudaStream_t st);

}  // namespace gks

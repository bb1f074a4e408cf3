// C ABI of the GB300 gas-kinetic solver: mesh and solver lifetime, state transfer, residual,
// two-stage fourth-order stepping and the time-step bound.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "gks_device.cuh"

using namespace gks;

namespace {
thread_local std::string g_mesh_err;

template <class T>
cudaError_t dalloc(T** p, int64_t n) {
  *p = nullptr;
  if (n <= 0) return cudaSuccess;
  return cudaMalloc((void**)p, sizeof(T) * (size_t)n);
}
template <class T>
cudaError_t upload(T** p, const std::vector<T>& v, cudaStream_t st) {
  cudaError_t e = dalloc(p, (int64_t)v.size());
  if (e != cudaSuccess || v.empty()) return e;
  return cudaMemcpyAsync(*p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, st);
}
}  // namespace

void gks::set_global_error(const char* msg) { g_mesh_err = msg ? msg : ""; }

struct gks_solver {
  gks_params prm;
  cudaStream_t st = nullptr;
  int device = 0;
  DevMesh m;
  Geo64 g;
  GeoR<double> gd;
  GeoR<float> gf;
  bool mixed = false;
  bool fp64upd = false;     // GKS_PREC_MIXED_FP64UPD: Q (FP64) is the master state of the steps
  int dbg_wait_tries = 0;   // gks_debug_recon_wait
  int dbg_withhold = 0;
  // buffers (internal order)
  // The state lives in the gather copy QA (FP64 values, or float-float pairs on the FP32 path);
  // Q is its FP64 [5][nc] form, refreshed from QA when a call needs it (q_stale after steps).
  double* Q = nullptr;      // [5][nc]
  bool q_stale = false;
  double* Qs = nullptr;     // staging for the residual calls
  double* L = nullptr;      // stage-1 L, Lt [5][nc]: 8 bytes per value (FP64, or a float-float
  double* Lt = nullptr;     // pair on the FP32 path)
  double* tmp = nullptr;    // staging in caller order [5][nc]
  double* tmp2 = nullptr;   // second staging buffer
  void* poly = nullptr;     // [nc][kPolyStride] in R
  void* fface = nullptr;    // [nf][kFaceStride] in R
  void* QA = nullptr;       // gather copy of Q (Lay<R>::gq values per cell)
  void* QsA = nullptr;      // gather copy of the stage state
  ForkJoin fj;             // concurrent reconstruction ranges
  // implicit step (allocated on the first gks_step_implicit call), precision R:
  bool imp_ready = false;
  void* jfn = nullptr;      // [nf][4] unit normal out of the owner, area
  void* jR = nullptr;       // [5][nc] |Omega| Res
  void* jD = nullptr;       // [nc] Jacobi diagonal
  void* jhrs = nullptr;     // [cf entries] r_f S_f / 2
  void* jdQ[2] = {nullptr, nullptr};  // [5][nc] Jacobi iterates
  int* flag = nullptr;      // device status bits
  int* bad_cell = nullptr;
  double* dt_part = nullptr;
  double* dt_out = nullptr;
  double* h_dt = nullptr;   // pinned host scalar
  std::vector<void*> owned;
  std::string err;
  // adjoint (allocated on the first gks_residual_vjp call)
  bool vjp_ready = false;
  GeoR<double> gv;             // FP64 geometry (the solver's own in FP64 mode)
  double* vQ = nullptr;        // internal-order state [5][nc]
  double* vQA = nullptr;       // its FP64 gather copy [nc][6]
  double* vpoly = nullptr;     // FP64 polynomials [nc][kPolyStride]
  double* vgL = nullptr;       // internal-order cotangents [5][nc]
  double* vgLt = nullptr;
  double* vgpf = nullptr;      // per face, both sides: polynomial cotangents [nf][2][kPolyStride]
  double* vgpc = nullptr;      // per cell polynomial cotangents [nc][kPolyStride]
  double* vgdq = nullptr;      // per stencil entry (tile layout) [slots][5][32]
  double* vgq0 = nullptr;      // [5][nc]
  double* vgQ = nullptr;       // [5][nc]
  int32_t* rs_ptr = nullptr;   // reverse stencil
  int32_t* rs_pos = nullptr;
  // optional per-kernel event timing
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_used;
  cudaEvent_t take_event() {
    if (!ev_pool.empty()) {
      cudaEvent_t e = ev_pool.back();
      ev_pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  // record a start event for kernel kind k; returns the index to close
  int tick(int kind) {
    if (!timing) return -1;
    cudaEvent_t a = take_event(), b = take_event();
    cudaEventRecord(a, st);
    ev_used.push_back({kind, {a, b}});
    return (int)ev_used.size() - 1;
  }
  void tock(int idx) {
    if (idx >= 0) cudaEventRecord(ev_used[idx].second.second, st);
  }

  gks_status fail(gks_status s, const std::string& msg) {
    err = msg;
    return s;
  }
  gks_status cuda_fail(cudaError_t e, const char* where) {
    err = std::string(where) + ": " + cudaGetErrorString(e);
    return GKS_E_CUDA;
  }
};

namespace {

template <class T>
cudaError_t salloc(gks_solver* s, T** p, int64_t n) {
  cudaError_t e = dalloc(p, n);
  if (e == cudaSuccess && *p) s->owned.push_back((void*)*p);
  return e;
}
template <class T>
cudaError_t supload(gks_solver* s, T** p, const std::vector<T>& v) {
  cudaError_t e = upload(p, v, s->st);
  if (e == cudaSuccess && *p) s->owned.push_back((void*)*p);
  return e;
}

template <class R>
KParams<R> kparams(const gks_params& p) {
  KParams<R> k;
  k.gamma = (R)p.gamma;
  k.K = (R)((5.0 - 3.0 * p.gamma) / (p.gamma - 1.0));
  k.mu = (R)p.mu;
  k.tau_eps = (R)p.tau_eps;
  k.tau_C = (R)p.tau_C;
  k.pr_fix = (R)(1.0 / p.Pr - 1.0);
  k.flux_mode = p.flux_mode;
  k.tau_model = p.tau_model;
  k.weno_gamma = (R)p.weno_gamma;
  k.weno_eps = (R)p.weno_eps;
  k.weno_pow = p.weno_pow;
  k.T_ref = (R)p.T_ref;
  k.mu_pow = (R)p.mu_pow;
  k.gp_fallback = p.gp_fallback != 0;
  return k;
}

// The precision-R geometry arrays (every field of GeoR<R>).
template <class R>
cudaError_t alloc_geo_arrays(gks_solver* s, GeoR<R>& g) {
  const int64_t nc = s->m.nc, nf = s->m.nf;
  cudaError_t e;
  if ((e = salloc(s, &g.Ap, 9 * (int64_t)kTile * s->m.n_tslots)) != cudaSuccess) return e;
  if ((e = salloc(s, &g.Bp, 4 * (int64_t)kTile * s->m.n_tsb)) != cudaSuccess) return e;
  if ((e = salloc(s, &g.mom, 6 * nc)) != cudaSuccess) return e;
  if ((e = salloc(s, &g.h, nc)) != cudaSuccess) return e;
  if ((e = salloc(s, &g.fgp, 40 * nf)) != cudaSuccess) return e;
  return salloc(s, &g.ivol, (sizeof(R) == 4 ? 2 : 1) * nc);
}

template <class R>
gks_status alloc_geo(gks_solver* s, GeoR<R>& g) {
  const int64_t nc = s->m.nc, nf = s->m.nf;
  cudaError_t e;
  if ((e = alloc_geo_arrays(s, g)) != cudaSuccess) return s->cuda_fail(e, "alloc geometry");
  R* poly = nullptr;
  R* ff = nullptr;
  R* qa = nullptr;
  R* qsa = nullptr;
  if ((e = salloc(s, &poly, (int64_t)kPolyStride * nc)) != cudaSuccess) return s->cuda_fail(e, "alloc poly");
  if ((e = salloc(s, &ff, (int64_t)kFaceStride * nf)) != cudaSuccess) return s->cuda_fail(e, "alloc face flux");
  const int64_t nq = nc + s->m.ng;  // cells and wall ghost slots
  if ((e = salloc(s, &qa, (int64_t)Lay<R>::gq * nq)) != cudaSuccess) return s->cuda_fail(e, "alloc gather copy");
  if ((e = salloc(s, &qsa, (int64_t)Lay<R>::gq * nq)) != cudaSuccess) return s->cuda_fail(e, "alloc gather copy");
  s->poly = poly;
  s->fface = ff;
  s->QA = qa;
  s->QsA = qsa;
  return GKS_OK;
}

template <class R>
void precompute_r(gks_solver* s, GeoR<R>& g) {
  launch_geom_faces<R>(s->m, s->g, g, s->st);
  launch_geom_hdt(s->m, s->g, s->st);
  launch_geom_ls<R>(s->m, s->g, g, s->flag, s->bad_cell, s->st);
  launch_cast_cells<R>(s->m, s->g, g, s->st);
}

// One residual evaluation: recon (from the gather copy QinA) -> flux -> face sums: the FP64
// residual (mode 0) or stage `mode` of the update.
template <class R>
void residual_r(gks_solver* s, GeoR<R>& g, const void* QinA, double dt, int mode, double* L,
                double* Lt) {
  KParams<R> kp = kparams<R>(s->prm);
  kp.wait_tries = s->dbg_wait_tries;
  kp.withhold = s->dbg_withhold;
  int t = s->tick(0);
  launch_recon<R>(s->m, g, kp, (const R*)QinA, (R*)s->poly, s->flag, s->st, &s->fj);
  s->tock(t);
  t = s->tick(1);
  launch_flux<R>(s->m, g, kp, (const R*)s->poly, (const R*)QinA, dt, (R*)s->fface, s->flag,
                 s->st);
  s->tock(t);
  t = s->tick(2);
  if (mode == 0)
    launch_gather<R>(s->m, s->g, (const R*)s->fface, L, Lt, s->st);
  else
    launch_stage<R>(s->m, g, (const R*)s->fface, mode, dt, L, Lt, (R*)s->QA, (R*)s->QsA,
                    s->flag, s->st, s->fp64upd ? s->Q : nullptr, s->g.ivol);
  s->tock(t);
}

void residual_any(gks_solver* s, const void* QinA, double dt, int mode, double* L, double* Lt) {
  if (s->mixed)
    residual_r<float>(s, s->gf, QinA, dt, mode, L, Lt);
  else
    residual_r<double>(s, s->gd, QinA, dt, mode, L, Lt);
}

// Caller-order state -> internal order (dst) and its gather copy (gq).
void permute_in_any(gks_solver* s, const double* src, double* dst, void* gq) {
  if (s->mixed)
    launch_permute_in<float>(s->m.nc, s->m.perm, src, dst, (float*)gq, s->st);
  else
    launch_permute_in<double>(s->m.nc, s->m.perm, src, dst, (double*)gq, s->st);
}

// Refresh the FP64 form of the state from its gather copy after steps.
void sync_q(gks_solver* s) {
  if (!s->q_stale) return;
  if (s->mixed)
    launch_unpack<float>(s->m.nc, (const float*)s->QA, s->Q, s->st);
  else
    launch_unpack<double>(s->m.nc, (const double*)s->QA, s->Q, s->st);
  s->q_stale = false;
}

gks_status read_flag(gks_solver* s, int* out) {
  cudaError_t e = cudaMemcpyAsync(s->h_dt, s->flag, sizeof(int), cudaMemcpyDeviceToHost, s->st);
  if (e != cudaSuccess) return s->cuda_fail(e, "status copy");
  e = cudaStreamSynchronize(s->st);
  if (e != cudaSuccess) return s->cuda_fail(e, "stream synchronise");
  std::memcpy(out, s->h_dt, sizeof(int));
  return GKS_OK;
}

gks_status check_and_clear(gks_solver* s) {
  int f = 0;
  gks_status r = read_flag(s, &f);
  if (r != GKS_OK) return r;
  if (f) {
    cudaMemsetAsync(s->flag, 0, sizeof(int), s->st);
    if (f & kErrNonphysical)
      return s->fail(GKS_E_NONPHYSICAL, "non-physical state (rho <= 0, p <= 0 or NaN)");
    if (f & kErrTimeout)
      return s->fail(GKS_E_TIMEOUT, "an asynchronous copy did not complete within its wait limit");
    return s->fail(GKS_E_CUDA, "device status " + std::to_string(f));
  }
  return GKS_OK;
}

// Ghost slots of moving no-slip walls (DevMesh::ng). The flow variables of a stencil image are
// the wall maps of the planes it was reflected across, applied in order (Section 2: ghost
// variables from the boundary condition): slip, m_axis -> -m_axis; no-slip with velocity U_w,
// rho -> rho, m -> 2 U_w rho - m, E -> E + 2 |U_w|^2 rho - 2 U_w . m (same density and
// pressure). The composition is kept as rho -> rho, m_j -> s_j m_j + a_j rho,
// E -> E + b rho + c . m. Entries whose map is a pure sign change keep their flip bits; the
// others point at a ghost slot nc + g (one per source cell and plane sequence).
struct WallMap {
  double s[3] = {1, 1, 1}, a[3] = {0, 0, 0}, b = 0, c[3] = {0, 0, 0};
};
WallMap wall_map_of(const HostMesh& h, const gks_params& p, uint8_t code) {
  WallMap M;
  for (int k = 0; k < 2; ++k) {
    const int w = ((code >> (3 * k)) & 7) - 1;
    if (w < 0) break;
    const int ax = w % 3;
    WallMap W;
    if (h.bc[ax] == GKS_BC_REFLECT) {
      W.s[ax] = -1;
    } else {
      const double* uw = p.wall_u[w];
      W.s[0] = W.s[1] = W.s[2] = -1;
      W.b = 2.0 * (uw[0] * uw[0] + uw[1] * uw[1] + uw[2] * uw[2]);
      for (int j = 0; j < 3; ++j) {
        W.a[j] = 2.0 * uw[j];
        W.c[j] = -2.0 * uw[j];
      }
    }
    WallMap C;  // W after M
    C.b = M.b + W.b;
    for (int j = 0; j < 3; ++j) {
      C.s[j] = W.s[j] * M.s[j];
      C.a[j] = W.s[j] * M.a[j] + W.a[j];
      C.c[j] = M.c[j] + M.s[j] * W.c[j];
      C.b += W.c[j] * M.a[j];
    }
    M = C;
  }
  return M;
}
bool wall_map_is_signs(const WallMap& M) {
  if (M.b != 0.0) return false;
  for (int j = 0; j < 3; ++j)
    if (M.a[j] != 0.0 || M.c[j] != 0.0) return false;
  return true;
}
// Patches the tile entries (t_idx) and fills the ghost tables; false if the slots do not fit
// the entry's cell field.
bool build_wall_ghosts(const HostMesh& h, const gks_params& p, std::vector<int32_t>& tidx,
                       std::vector<int32_t>& gsrc, std::vector<double>& gmap,
                       std::vector<float>& gmapf, std::vector<uint8_t>& gchain) {
  tidx = h.t_idx;
  gsrc.clear();
  gmap.clear();
  gmapf.clear();
  gchain.clear();
  bool any = false;
  for (int a = 0; a < 3; ++a) any = any || h.bc[a] == GKS_BC_NOSLIP || h.bc[a] == GKS_BC_FARFIELD;
  if (!any) return true;
  const int64_t nc = h.n_cells;
  std::map<int64_t, int32_t> slot_of;  // (src << 8 | plane code) -> slot
  for (int64_t t = 0; t < h.n_tiles; ++t)
    for (int l = 0; l < kTile; ++l) {
      const int64_t c = t * kTile + l;
      if (c >= nc) continue;
      const int Kc = h.st_ptr[c + 1] - h.st_ptr[c];
      for (int k = 0; k < Kc; ++k) {
        const int64_t e = h.st_ptr[c] + k;
        const uint8_t code = h.st_walls[e];
        if (!code) continue;
        bool far = false;
        for (int q = 0; q < 2; ++q) {
          const int w = ((code >> (3 * q)) & 7) - 1;
          far = far || (w >= 0 && h.bc[w % 3] == GKS_BC_FARFIELD);
        }
        const WallMap M = far ? WallMap() : wall_map_of(h, p, code);
        if (!far && wall_map_is_signs(M)) continue;
        const int32_t src = h.st_idx[e] & kCellMask;
        const int64_t key = ((int64_t)src << 8) | code;
        auto it = slot_of.find(key);
        int32_t g;
        if (it == slot_of.end()) {
          g = (int32_t)gsrc.size();
          slot_of.emplace(key, g);
          gsrc.push_back(src);
          gchain.push_back(far ? code : 0);
          const double v[10] = {M.s[0], M.s[1], M.s[2], M.a[0], M.a[1], M.a[2], M.b,
                                M.c[0], M.c[1], M.c[2]};
          for (double x : v) {
            gmap.push_back(x);
            const float hi = (float)x;
            gmapf.push_back(hi);
            gmapf.push_back((float)(x - (double)hi));
          }
        } else {
          g = it->second;
        }
        if (nc + g > (int64_t)kCellMask) return false;
        tidx[((size_t)h.t_st[t] + k) * kTile + l] = (int32_t)(nc + g);
      }
    }
  return true;
}

bool valid_params(const gks_params* p, std::string& why) {
  if (!(p->gamma > 1.0 && p->gamma < 5.0 / 3.0 + 1e-12)) { why = "gamma must lie in (1, 5/3]"; return false; }
  if (!(p->mu >= 0.0)) { why = "mu must be >= 0"; return false; }
  if (!(p->Pr > 0.0)) { why = "Pr must be > 0"; return false; }
  if (p->Pr != 1.0 && p->flux_mode != GKS_FLUX_SMOOTH) {
    why = "the Prandtl-number correction is implemented for the smooth flux only";
    return false;
  }
  if (p->flux_mode != GKS_FLUX_SMOOTH && p->flux_mode != GKS_FLUX_FULL) { why = "flux_mode"; return false; }
  if (p->tau_model < GKS_TAU_ZERO || p->tau_model > GKS_TAU_POWER_LAW) { why = "tau_model"; return false; }
  if (p->tau_model == GKS_TAU_POWER_LAW && !(p->T_ref > 0.0 && std::isfinite(p->mu_pow))) {
    why = "the power law needs T_ref > 0 and a finite exponent";
    return false;
  }
  for (int w = 0; w < 6; ++w)
    if (!(std::isfinite(p->wall_u[w][0]) && std::isfinite(p->wall_u[w][1]) &&
          std::isfinite(p->wall_u[w][2]) && std::isfinite(p->wall_T[w]))) {
      why = "wall velocity and temperature must be finite";
      return false;
    }
  for (int w = 0; w < 6; ++w)
    if (!(p->farfield[w][0] > 0.0 && p->farfield[w][4] > 0.0 &&
          std::isfinite(p->farfield[w][0]) && std::isfinite(p->farfield[w][4]) &&
          std::isfinite(p->farfield[w][1]) && std::isfinite(p->farfield[w][2]) &&
          std::isfinite(p->farfield[w][3]))) {
      why = "a far-field state needs rho > 0, p > 0 and a finite velocity";
      return false;
    }
  if (!(p->weno_gamma > 0.0 && p->weno_gamma * 8 < 1.0)) { why = "weno_gamma must lie in (0, 1/8)"; return false; }
  if (!(p->weno_eps > 0.0)) { why = "weno_eps must be > 0"; return false; }
  if (p->weno_pow < 1 || p->weno_pow > 4) { why = "weno_pow must be 1..4"; return false; }
  if (p->precision != GKS_PREC_FP64 && p->precision != GKS_PREC_MIXED &&
      p->precision != GKS_PREC_MIXED_FP64UPD) {
    why = "precision";
    return false;
  }
  return true;
}

template <class R>
gks_status step_implicit_r(gks_solver* s, GeoR<R>& g, double dt, int nsteps, int kmax) {
  const int64_t nc = s->m.nc, nf = s->m.nf;
  cudaError_t e = cudaSuccess;
  if (!s->imp_ready) {
    R *fn = nullptr, *rv = nullptr, *d = nullptr, *hrs = nullptr, *a = nullptr, *b = nullptr;
    if ((e = salloc(s, &fn, 4 * nf)) != cudaSuccess || (e = salloc(s, &rv, 5 * nc)) != cudaSuccess ||
        (e = salloc(s, &d, nc)) != cudaSuccess || (e = salloc(s, &hrs, s->m.ncf)) != cudaSuccess ||
        (e = salloc(s, &a, 5 * nc)) != cudaSuccess || (e = salloc(s, &b, 5 * nc)) != cudaSuccess)
      return s->cuda_fail(e, "implicit buffers");
    s->jfn = fn;
    s->jR = rv;
    s->jD = d;
    s->jhrs = hrs;
    s->jdQ[0] = a;
    s->jdQ[1] = b;
    launch_face_normals<R>(s->m, fn, s->st);
    s->imp_ready = true;
  }
  KParams<R> kp = kparams<R>(s->prm);
  kp.wait_tries = s->dbg_wait_tries;
  kp.withhold = s->dbg_withhold;
  R* dq[2] = {(R*)s->jdQ[0], (R*)s->jdQ[1]};
  for (int n = 0; n < nsteps; ++n) {
    int t = s->tick(0);
    launch_recon<R>(s->m, g, kp, (const R*)s->QA, (R*)s->poly, s->flag, s->st, &s->fj);
    s->tock(t);
    t = s->tick(1);
    launch_flux<R>(s->m, g, kp, (const R*)s->poly, (const R*)s->QA, dt, (R*)s->fface, s->flag,
                   s->st);
    s->tock(t);
    t = s->tick(2);
    launch_jacobi_init<R>(s->m, (const R*)s->fface, (const R*)s->jfn, s->g.vol, dt,
                          (const R*)s->QA, (R*)s->jR, (R*)s->jD, (R*)s->jhrs, dq[0], kp,
                          s->st);
    for (int it = 1; it <= kmax; ++it)
      launch_jacobi_sweep<R>(s->m, (const R*)s->jfn, (const R*)s->QA, (const R*)s->jR,
                             (const R*)s->jD, (const R*)s->jhrs, dq[(it - 1) & 1], dq[it & 1],
                             it == kmax, (R*)s->QsA, kp, s->flag, s->st);
    s->tock(t);
    std::swap(s->QA, s->QsA);  // Q^{n+1} was written to the other gather copy
  }
  if (nsteps > 0) s->q_stale = true;
  e = cudaGetLastError();
  return e == cudaSuccess ? GKS_OK : s->cuda_fail(e, "implicit step launch");
}

}  // namespace

extern "C" {

void gks_params_default(gks_params* p) {
  if (!p) return;
  p->gamma = 1.4;
  p->mu = 0.0;
  p->Pr = 1.0;
  p->flux_mode = GKS_FLUX_SMOOTH;
  p->tau_model = GKS_TAU_ZERO;
  p->tau_eps = 0.01;
  p->tau_C = 1.0;
  p->weno_gamma = 0.0125;
  p->weno_eps = 1e-8;
  p->weno_pow = 1;
  p->precision = GKS_PREC_FP64;
  p->T_ref = 1.0;
  p->mu_pow = 0.7;
  for (int w = 0; w < 6; ++w) {
    p->wall_u[w][0] = p->wall_u[w][1] = p->wall_u[w][2] = 0.0;
    p->wall_T[w] = 0.0;
  }
  for (int w = 0; w < 6; ++w) {
    p->farfield[w][0] = 1.0;
    p->farfield[w][1] = p->farfield[w][2] = p->farfield[w][3] = 0.0;
    p->farfield[w][4] = 1.0 / 1.4;
  }
  p->gp_fallback = 0;
}

gks_status gks_mesh_create(int64_t n_nodes, const double* xyz, int64_t n_cells,
                           const int8_t* cell_type, const int64_t* cell_nodes, const int bc[3],
                           const double lo[3], const double hi[3], gks_mesh** out) {
  return gks_mesh_create_ex(n_nodes, xyz, n_cells, cell_type, cell_nodes, bc, lo, hi, nullptr,
                            out);
}

gks_status gks_mesh_create_ex(int64_t n_nodes, const double* xyz, int64_t n_cells,
                              const int8_t* cell_type, const int64_t* cell_nodes, const int bc[3],
                              const double lo[3], const double hi[3],
                              const gks_mesh_options* opt, gks_mesh** out) {
  if (!out) return GKS_E_INVAL;
  *out = nullptr;
  const int reorder = opt ? opt->reorder : GKS_REORDER_MORTON;
  const int min_stencil = opt ? opt->min_stencil : 0;
  gks_mesh* m = new (std::nothrow) gks_mesh;
  if (!m) return GKS_E_NOMEM;
  gks_status st;
  try {
    st = build_host_mesh(n_nodes, xyz, n_cells, cell_type, cell_nodes, bc, lo, hi, reorder,
                         min_stencil, m->h, g_mesh_err);
  } catch (const std::bad_alloc&) {
    g_mesh_err = "host allocation failed";
    st = GKS_E_NOMEM;
  }
  if (st != GKS_OK) {
    delete m;
    return st;
  }
  *out = m;
  return GKS_OK;
}

gks_status gks_mesh_counts(const gks_mesh* m, int64_t* n_cells, int64_t* n_faces,
                           int64_t* n_stencil) {
  if (!m) return GKS_E_INVAL;
  if (n_cells) *n_cells = m->h.n_cells;
  if (n_faces) *n_faces = m->h.n_faces;
  if (n_stencil) *n_stencil = (int64_t)m->h.st_idx.size();
  return GKS_OK;
}

const char* gks_mesh_last_error(void) { return g_mesh_err.c_str(); }

void gks_mesh_destroy(gks_mesh* m) { delete m; }

gks_status gks_init(const gks_mesh* mesh, const gks_params* p, void* stream, gks_solver** out) {
  if (!out) return GKS_E_INVAL;
  *out = nullptr;
  if (!mesh || !p) return GKS_E_INVAL;
  std::string why;
  if (!valid_params(p, why)) {
    g_mesh_err = why;
    return GKS_E_INVAL;
  }
  gks_solver* s = new (std::nothrow) gks_solver;
  if (!s) return GKS_E_NOMEM;
  s->prm = *p;
  s->st = (cudaStream_t)stream;
  s->mixed = p->precision == GKS_PREC_MIXED || p->precision == GKS_PREC_MIXED_FP64UPD;
  s->fp64upd = p->precision == GKS_PREC_MIXED_FP64UPD;
  cudaGetDevice(&s->device);
  const HostMesh& h = mesh->h;
  DevMesh& m = s->m;
  m.nc = h.n_cells;
  m.nf = h.n_faces;
  m.nst = (int64_t)h.st_idx.size();
  m.nsb = h.sb_ptr.back();
  for (int64_t i = 0; i < h.n_cells; ++i) m.kmax = std::max(m.kmax, h.st_ptr[i + 1] - h.st_ptr[i]);
  cudaError_t e = cudaSuccess;
  auto bad = [&](const char* what) {
    gks_status r = e == cudaErrorMemoryAllocation ? GKS_E_NOMEM : GKS_E_CUDA;
    g_mesh_err = std::string(what) + ": " + cudaGetErrorString(e);
    gks_destroy(s);
    return r;
  };
  if ((e = supload(s, &m.perm, h.perm)) != cudaSuccess) return bad("upload");
  if ((e = supload(s, &m.type, h.type)) != cudaSuccess) return bad("upload");
  if ((e = supload(s, &m.cell_x, h.cell_x)) != cudaSuccess) return bad("upload");
  if ((e = supload(s, &m.f_owner, h.f_owner)) != cudaSuccess) return bad("upload");
  if ((e = supload(s, &m.f_nb, h.f_nb)) != cudaSuccess) return bad("upload");
  if ((e = supload(s, &m.f_wall, h.f_wall)) != cudaSuccess) return bad("upload");
  if ((e = supload(s, &m.f_vert, h.f_vert)) != cudaSuccess) return bad("upload");
  if ((e = supload(s, &m.f_shift, h.f_shift)) != cudaSuccess) return bad("upload");
  if ((e = supload(s, &m.cf_ptr, h.cf_ptr)) != cudaSuccess) return bad("upload");
  if ((e = supload(s, &m.cf_idx, h.cf_idx)) != cudaSuccess) return bad("upload");
  m.ncf = (int64_t)h.cf_idx.size();
  if ((e = supload(s, &m.st_ptr, h.st_ptr)) != cudaSuccess) return bad("upload");
  if ((e = supload(s, &m.st_idx, h.st_idx)) != cudaSuccess) return bad("upload");
  if ((e = supload(s, &m.st_xf, h.st_xf)) != cudaSuccess) return bad("upload");
  if ((e = supload(s, &m.st_sub, h.st_sub)) != cudaSuccess) return bad("upload");
  if ((e = supload(s, &m.n_sub, h.n_sub)) != cudaSuccess) return bad("upload");
  if ((e = supload(s, &m.sb_ptr, h.sb_ptr)) != cudaSuccess) return bad("upload");
  if ((e = supload(s, &m.sub_cnt, h.sub_cnt)) != cudaSuccess) return bad("upload");
  m.n_tiles = h.n_tiles;
  m.n_tslots = h.t_st.back();
  m.n_tsb = h.t_sb.back();
  if ((e = supload(s, &m.t_K, h.t_K)) != cudaSuccess) return bad("upload");
  if ((e = supload(s, &m.t_cnt, h.t_cnt)) != cudaSuccess) return bad("upload");
  if ((e = supload(s, &m.t_st, h.t_st)) != cudaSuccess) return bad("upload");
  if ((e = supload(s, &m.t_sb, h.t_sb)) != cudaSuccess) return bad("upload");
  {
    std::vector<int32_t> tidx, gsrc;
    std::vector<double> gmap;
    std::vector<float> gmapf;
    std::vector<uint8_t> gchain;
    if (!build_wall_ghosts(h, *p, tidx, gsrc, gmap, gmapf, gchain)) {
      g_mesh_err = "too many wall ghost cells for the stencil entry format";
      gks_destroy(s);
      return GKS_E_MESH;
    }
    if ((e = supload(s, &m.t_idx, tidx)) != cudaSuccess) return bad("upload");
    std::vector<double> w64(6 * kPlaneStride, 0.0);
    std::vector<float> w32(6 * kPlaneStride);
    for (int w = 0; w < 6; ++w) {
      double* t = w64.data() + kPlaneStride * w;
      for (int a = 0; a < 3; ++a) t[a] = p->wall_u[w][a];
      t[3] = p->wall_T[w];
      for (int v = 0; v < 5; ++v) t[4 + v] = p->farfield[w][v];
    }
    for (size_t k = 0; k < w64.size(); ++k) w32[k] = (float)w64[k];
    if ((e = supload(s, &m.wall64, w64)) != cudaSuccess) return bad("upload");
    if ((e = supload(s, &m.wall32, w32)) != cudaSuccess) return bad("upload");
    m.ng = (int64_t)gsrc.size();
    if (m.ng > 0) {
      if ((e = supload(s, &m.g_src, gsrc)) != cudaSuccess) return bad("upload");
      if ((e = supload(s, &m.g_map, gmap)) != cudaSuccess) return bad("upload");
      if ((e = supload(s, &m.g_mapf, gmapf)) != cudaSuccess) return bad("upload");
      if ((e = supload(s, &m.g_chain, gchain)) != cudaSuccess) return bad("upload");
    }
    m.bcs = h.bc[0] | (h.bc[1] << 2) | (h.bc[2] << 4);
  }
  // tile ranges by the kind of each tile's first cell (at most one per kind: cells are ordered
  // by kind first); a new range is opened only while slots remain, else the last one grows
  for (int64_t t = 0; t < h.n_tiles; ++t) {
    TileRanges& r = m.rr;
    const int kind = h.type[t * kTile];
    if (r.n == 0 || (kind != h.type[r.t0[r.n - 1] * kTile] && r.n < kMaxTileRanges)) {
      r.t0[r.n] = t;
      r.t1[r.n] = t;
      r.K[r.n] = r.S[r.n] = r.M[r.n] = 0;
      ++r.n;
    }
    int S = 0, M = 0;
    for (int q = 0; q < kMaxSub; ++q) {
      const int c = (int)((h.t_cnt[t] >> (8 * q)) & 0xffu);
      S += c;
      if (c) M = q + 1;
    }
    r.t1[r.n - 1] = t + 1;
    r.K[r.n - 1] = std::max(r.K[r.n - 1], h.t_K[t]);
    r.S[r.n - 1] = std::max(r.S[r.n - 1], S);
    r.M[r.n - 1] = std::max(r.M[r.n - 1], M);
  }
  // a range is uniform when all its tiles match the first one's stencil size and sub-stencil
  // counts (then t_st and t_sb grow by K and S per tile, and the kernel needs no table loads)
  for (int k = 0; k < m.rr.n; ++k) {
    TileRanges& r = m.rr;
    const int64_t a = r.t0[k];
    int S0 = 0;
    for (int q = 0; q < kMaxSub; ++q) S0 += (int)((h.t_cnt[a] >> (8 * q)) & 0xffu);
    bool uni = r.t1[k] > a;
    for (int64_t t = a; t < r.t1[k] && uni; ++t)
      uni = h.t_K[t] == h.t_K[a] && h.t_cnt[t] == h.t_cnt[a] &&
            (int64_t)h.t_st[t] == (int64_t)h.t_st[a] + (t - a) * h.t_K[a] &&
            (int64_t)h.t_sb[t] == (int64_t)h.t_sb[a] + (t - a) * S0;
    r.uni[k] = uni ? 1 : 0;
    r.cnt[k] = h.t_cnt[a];
    r.st0[k] = h.t_st[a];
    r.sb0[k] = h.t_sb[a];
  }
  // auxiliary streams for the concurrent reconstruction ranges (serial if unavailable)
  if (m.rr.n > 1 && cudaEventCreateWithFlags(&s->fj.fork, cudaEventDisableTiming) == cudaSuccess) {
    for (int k = 0; k < m.rr.n - 1; ++k) {
      if (cudaStreamCreateWithFlags(&s->fj.aux[k], cudaStreamNonBlocking) != cudaSuccess) break;
      if (cudaEventCreateWithFlags(&s->fj.join[k], cudaEventDisableTiming) != cudaSuccess) {
        cudaStreamDestroy(s->fj.aux[k]);
        break;
      }
      s->fj.n = k + 1;
    }
  }
  cudaGetLastError();  // a failed optional creation leaves no sticky error
  if ((e = supload(s, &s->rs_ptr, h.rs_ptr)) != cudaSuccess) return bad("upload");
  if ((e = supload(s, &s->rs_pos, h.rs_pos)) != cudaSuccess) return bad("upload");
  const int64_t nc = m.nc, nf = m.nf;
  if ((e = salloc(s, &s->g.vol, nc)) != cudaSuccess) return bad("alloc");
  if ((e = salloc(s, &s->g.ivol, nc)) != cudaSuccess) return bad("alloc");
  if ((e = salloc(s, &s->g.cen, 3 * nc)) != cudaSuccess) return bad("alloc");
  if ((e = salloc(s, &s->g.h, nc)) != cudaSuccess) return bad("alloc");
  if ((e = salloc(s, &s->g.mom, 6 * nc)) != cudaSuccess) return bad("alloc");
  if ((e = salloc(s, &s->g.hdt, nc)) != cudaSuccess) return bad("alloc");
  if ((e = salloc(s, &s->g.farea, nf)) != cudaSuccess) return bad("alloc");
  if ((e = salloc(s, &s->Q, 5 * nc)) != cudaSuccess) return bad("alloc");
  if ((e = salloc(s, &s->Qs, 5 * nc)) != cudaSuccess) return bad("alloc");
  if ((e = salloc(s, &s->L, 5 * nc)) != cudaSuccess) return bad("alloc");
  if ((e = salloc(s, &s->Lt, 5 * nc)) != cudaSuccess) return bad("alloc");
  if ((e = salloc(s, &s->tmp, 5 * nc)) != cudaSuccess) return bad("alloc");
  if ((e = salloc(s, &s->tmp2, 5 * nc)) != cudaSuccess) return bad("alloc");
  if ((e = salloc(s, &s->flag, 2)) != cudaSuccess) return bad("alloc");
  s->bad_cell = s->flag + 1;
  if ((e = salloc(s, &s->dt_part, dt_blocks(nc) + 1)) != cudaSuccess) return bad("alloc");
  s->dt_out = s->dt_part + dt_blocks(nc);
  if ((e = cudaMallocHost((void**)&s->h_dt, 16)) != cudaSuccess) return bad("alloc pinned");
  const int init_flags[2] = {0, 0x7fffffff};
  if ((e = cudaMemcpyAsync(s->flag, init_flags, sizeof(init_flags), cudaMemcpyHostToDevice, s->st)) !=
      cudaSuccess)
    return bad("memcpy");
  gks_status r = s->mixed ? alloc_geo(s, s->gf) : alloc_geo(s, s->gd);
  if (r != GKS_OK) {
    g_mesh_err = s->err;
    gks_destroy(s);
    return r;
  }
  launch_geom_cells(s->m, s->g, s->flag, s->st);
  if (s->mixed)
    precompute_r(s, s->gf);
  else
    precompute_r(s, s->gd);
  e = cudaGetLastError();
  if (e != cudaSuccess) return bad("precompute launch");
  int flags[2];
  e = cudaMemcpyAsync(flags, s->flag, sizeof(flags), cudaMemcpyDeviceToHost, s->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
  if (e != cudaSuccess) return bad("precompute");
  if (flags[0]) {
    gks_status code = (flags[0] & kErrInverted) ? GKS_E_MESH : GKS_E_SINGULAR;
    g_mesh_err = (flags[0] & kErrInverted) ? "inverted or degenerate cell"
                                           : "rank-deficient stencil at internal cell " +
                                                 std::to_string(flags[1]) + " (caller cell " +
                                                 std::to_string(h.perm[flags[1] < nc ? flags[1] : 0]) + ")";
    gks_destroy(s);
    return code;
  }
  *out = s;
  return GKS_OK;
}

gks_status gks_set_state(gks_solver* s, const double* Q) {
  if (!s || !Q) return GKS_E_INVAL;
  const int64_t nc = s->m.nc;
  cudaError_t e = cudaMemcpyAsync(s->tmp, Q, sizeof(double) * 5 * nc, cudaMemcpyDefault, s->st);
  if (e != cudaSuccess) return s->cuda_fail(e, "set_state copy");
  permute_in_any(s, s->tmp, s->Q, s->QA);
  s->q_stale = false;
  e = cudaGetLastError();
  return e == cudaSuccess ? GKS_OK : s->cuda_fail(e, "set_state");
}

gks_status gks_get_state(gks_solver* s, double* Q) {
  if (!s || !Q) return GKS_E_INVAL;
  const int64_t nc = s->m.nc;
  sync_q(s);
  launch_permute_out(nc, s->m.perm, s->Q, s->tmp, s->st);
  cudaError_t e = cudaMemcpyAsync(Q, s->tmp, sizeof(double) * 5 * nc, cudaMemcpyDefault, s->st);
  if (e != cudaSuccess) return s->cuda_fail(e, "get_state copy");
  e = cudaStreamSynchronize(s->st);
  return e == cudaSuccess ? GKS_OK : s->cuda_fail(e, "get_state");
}

gks_status gks_max_dt(gks_solver* s, double cfl, double* dt) {
  if (!s || !dt || !(cfl > 0)) return GKS_E_INVAL;
  sync_q(s);
  launch_check_state(s->m.nc, s->Q, s->prm.gamma, s->flag, s->st);
  const int nb = dt_blocks(s->m.nc);
  launch_dt(s->m.nc, s->Q, s->g.hdt, s->prm.gamma, s->prm.mu,
            s->prm.tau_model == GKS_TAU_POWER_LAW, s->prm.T_ref, s->prm.mu_pow, s->dt_part, nb,
            s->dt_out, s->st);
  gks_status r = check_and_clear(s);
  if (r != GKS_OK) return r;
  cudaError_t e = cudaMemcpyAsync(s->h_dt, s->dt_out, sizeof(double), cudaMemcpyDeviceToHost, s->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
  if (e != cudaSuccess) return s->cuda_fail(e, "max_dt");
  *dt = cfl * s->h_dt[0];
  return GKS_OK;
}

gks_status gks_step(gks_solver* s, double dt, int nsteps) {
  if (!s || !(dt > 0) || nsteps < 0) return GKS_E_INVAL;
  if (s->fp64upd) sync_q(s);  // after implicit steps the float-pair copy is the newer state
  for (int k = 0; k < nsteps; ++k) {
    // stage 1 on Q^n (QA): L, Lt kept, Q* to QsA; stage 2 on Q*: Q^{n+1} written into QA
    residual_any(s, s->QA, dt, 1, s->L, s->Lt);
    residual_any(s, s->QsA, dt, 2, s->L, s->Lt);
  }
  // the FP64-update mode writes its FP64 state in place; the others update the gather copy
  if (nsteps > 0 && !s->fp64upd) s->q_stale = true;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GKS_OK : s->cuda_fail(e, "step launch");
}

gks_status gks_debug_recon_wait(gks_solver* s, int wait_tries, int withhold_copies) {
  if (!s || wait_tries < 0) return GKS_E_INVAL;
  s->dbg_wait_tries = wait_tries;
  s->dbg_withhold = withhold_copies != 0;
  return GKS_OK;
}

gks_status gks_s2o4_stage(int64_t n, int stage, double dt, const double* Q, const double* L,
                          const double* Lt, const double* Lts, double* out, void* stream) {
  if (n < 0 || (stage != 1 && stage != 2) || !(dt > 0) || (n > 0 && (!Q || !L || !Lt || !out)) ||
      (n > 0 && stage == 2 && !Lts)) {
    set_global_error("gks_s2o4_stage: invalid argument");
    return GKS_E_INVAL;
  }
  if (n == 0) return GKS_OK;
  launch_s2o4_stage(n, stage, dt, Q, L, Lt, Lts, out, static_cast<cudaStream_t>(stream));
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_global_error((std::string("gks_s2o4_stage: ") + cudaGetErrorString(e)).c_str());
    return GKS_E_CUDA;
  }
  return GKS_OK;
}

gks_status gks_s2o4_stage_vjp(int64_t n, int stage, double dt, const double* g, double* gQ,
                              double* gL, double* gLt, double* gLts, void* stream) {
  if (n < 0 || (stage != 1 && stage != 2) || !(dt > 0) ||
      (n > 0 && (!g || !gQ || !gL || !gLt)) || (n > 0 && stage == 2 && !gLts)) {
    set_global_error("gks_s2o4_stage_vjp: invalid argument");
    return GKS_E_INVAL;
  }
  if (n == 0) return GKS_OK;
  launch_s2o4_stage_vjp(n, stage, dt, g, gQ, gL, gLt, gLts, static_cast<cudaStream_t>(stream));
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_global_error((std::string("gks_s2o4_stage_vjp: ") + cudaGetErrorString(e)).c_str());
    return GKS_E_CUDA;
  }
  return GKS_OK;
}

gks_status gks_step_implicit(gks_solver* s, double dt, int nsteps, int kmax) {
  if (!s || !(dt > 0) || nsteps < 0 || kmax < 1) return GKS_E_INVAL;
  return s->mixed ? step_implicit_r<float>(s, s->gf, dt, nsteps, kmax)
                  : step_implicit_r<double>(s, s->gd, dt, nsteps, kmax);
}

gks_status gks_check(gks_solver* s) {
  if (!s) return GKS_E_INVAL;
  return check_and_clear(s);
}

gks_status gks_residual(gks_solver* s, const double* Q, double dt, double* L, double* Lt) {
  if (!s || !Q || !L || !Lt || !(dt > 0)) return GKS_E_INVAL;
  const int64_t nc = s->m.nc;
  cudaError_t e = cudaMemcpyAsync(s->tmp, Q, sizeof(double) * 5 * nc, cudaMemcpyDefault, s->st);
  if (e != cudaSuccess) return s->cuda_fail(e, "residual copy");
  permute_in_any(s, s->tmp, s->Qs, s->QsA);
  launch_check_state(nc, s->Qs, s->prm.gamma, s->flag, s->st);
  residual_any(s, s->QsA, dt, 0, s->tmp, s->tmp2);
  // tmp, tmp2 hold L, Lt in internal order; write them out in caller order
  launch_permute_out(nc, s->m.perm, s->tmp, s->Qs, s->st);
  e = cudaMemcpyAsync(L, s->Qs, sizeof(double) * 5 * nc, cudaMemcpyDefault, s->st);
  if (e != cudaSuccess) return s->cuda_fail(e, "residual copy out");
  launch_permute_out(nc, s->m.perm, s->tmp2, s->tmp, s->st);
  e = cudaMemcpyAsync(Lt, s->tmp, sizeof(double) * 5 * nc, cudaMemcpyDefault, s->st);
  if (e != cudaSuccess) return s->cuda_fail(e, "residual copy out");
  e = cudaGetLastError();
  if (e != cudaSuccess) return s->cuda_fail(e, "residual launch");
  return check_and_clear(s);
}

gks_status gks_residual_vjp(gks_solver* s, const double* Q, double dt, const double* gL,
                            const double* gLt, double* gQ) {
  if (!s || !Q || !gL || !gLt || !gQ || !(dt > 0)) return GKS_E_INVAL;
  if (s->prm.Pr != 1.0) return s->fail(GKS_E_INVAL, "the VJP supports Pr = 1 only");
  const int64_t nc = s->m.nc, nf = s->m.nf;
  cudaError_t e = cudaSuccess;
  if (!s->vjp_ready) {
    if (s->mixed) {
      // FP64 geometry of its own (the FP32 path keeps only FP32 copies)
      GeoR<double>& g = s->gv;
      if ((e = alloc_geo_arrays(s, g)) != cudaSuccess) return s->cuda_fail(e, "vjp geometry");
      precompute_r(s, g);
    } else {
      s->gv = s->gd;
    }
    if ((e = salloc(s, &s->vQ, 5 * nc)) != cudaSuccess ||
        (e = salloc(s, &s->vQA, 6 * (nc + s->m.ng))) != cudaSuccess ||
        (e = salloc(s, &s->vpoly, (int64_t)kPolyStride * nc)) != cudaSuccess ||
        (e = salloc(s, &s->vgL, 5 * nc)) != cudaSuccess ||
        (e = salloc(s, &s->vgLt, 5 * nc)) != cudaSuccess ||
        (e = salloc(s, &s->vgpf, 2 * (int64_t)kPolyStride * nf)) != cudaSuccess ||
        (e = salloc(s, &s->vgpc, (int64_t)kPolyStride * nc)) != cudaSuccess ||
        (e = salloc(s, &s->vgdq, 5 * (int64_t)kTile * s->m.n_tslots)) != cudaSuccess ||
        (e = salloc(s, &s->vgq0, 5 * nc)) != cudaSuccess ||
        (e = salloc(s, &s->vgQ, 5 * nc)) != cudaSuccess)
      return s->cuda_fail(e, "vjp buffers");
    s->vjp_ready = true;
  }
  const size_t bytes = sizeof(double) * 5 * nc;
  // inputs to internal order
  if ((e = cudaMemcpyAsync(s->tmp, Q, bytes, cudaMemcpyDefault, s->st)) != cudaSuccess)
    return s->cuda_fail(e, "vjp copy");
  launch_permute_in<double>(nc, s->m.perm, s->tmp, s->vQ, s->vQA, s->st);
  launch_check_state(nc, s->vQ, s->prm.gamma, s->flag, s->st);
  if ((e = cudaMemcpyAsync(s->tmp, gL, bytes, cudaMemcpyDefault, s->st)) != cudaSuccess)
    return s->cuda_fail(e, "vjp copy");
  launch_permute_in<double>(nc, s->m.perm, s->tmp, s->vgL, (double*)nullptr, s->st);
  if ((e = cudaMemcpyAsync(s->tmp, gLt, bytes, cudaMemcpyDefault, s->st)) != cudaSuccess)
    return s->cuda_fail(e, "vjp copy");
  launch_permute_in<double>(nc, s->m.perm, s->tmp, s->vgLt, (double*)nullptr, s->st);
  // forward reconstruction in FP64, then the reverse passes
  const KParams<double> kp = kparams<double>(s->prm);
  launch_recon<double>(s->m, s->gv, kp, s->vQA, s->vpoly, s->flag, s->st);
  launch_vjp(s->m, s->g, s->gv, kp, s->vQA, s->vpoly, s->vgL, s->vgLt, dt, s->vgpf, s->vgpc,
             s->vgdq, s->vgq0, s->vgQ, s->rs_ptr, s->rs_pos, s->flag, s->st);
  launch_permute_out(nc, s->m.perm, s->vgQ, s->tmp, s->st);
  if ((e = cudaMemcpyAsync(gQ, s->tmp, bytes, cudaMemcpyDefault, s->st)) != cudaSuccess)
    return s->cuda_fail(e, "vjp copy out");
  e = cudaGetLastError();
  if (e != cudaSuccess) return s->cuda_fail(e, "vjp launch");
  return check_and_clear(s);
}

gks_status gks_cell_quadrature(gks_solver* s, double* xq, double* wq) {
  if (!s || !xq || !wq) return GKS_E_INVAL;
  const int64_t nc = s->m.nc;
  double* dx = nullptr;
  double* dw = nullptr;
  cudaError_t e = cudaMalloc((void**)&dx, sizeof(double) * 81 * nc);
  if (e == cudaSuccess) e = cudaMalloc((void**)&dw, sizeof(double) * 27 * nc);
  if (e == cudaSuccess) {
    launch_cell_quadrature(s->m, dx, dw, s->st);
    e = cudaMemcpyAsync(xq, dx, sizeof(double) * 81 * nc, cudaMemcpyDefault, s->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(wq, dw, sizeof(double) * 27 * nc, cudaMemcpyDefault, s->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
  }
  if (dx) cudaFree(dx);
  if (dw) cudaFree(dw);
  return e == cudaSuccess ? GKS_OK : s->cuda_fail(e, "cell quadrature");
}

gks_status gks_kernel_bytes(const gks_solver* s, double bytes[3]) {
  if (!s || !bytes) return GKS_E_INVAL;
  const double nc = (double)s->m.nc, nf = (double)s->m.nf;
  const double ncf = 2.0 * nf;  // each face appears in two cells
  const double r = s->mixed ? 4.0 : 8.0;
  const double ts = (double)kTile * s->m.n_tslots, tb = (double)kTile * s->m.n_tsb;
  // reconstruction: gather copy of Q (48 B per cell, own + stencil, once), tile counts and
  // offsets, interleaved stencil entries, pseudo-inverse rows and sub-stencil entries (with the
  // tile padding, 0.4 % on the hybrid mesh), cell moments and size, polynomial written
  bytes[0] = 48.0 * nc + 24.0 * (double)s->m.n_tiles + nc + 4.0 * ts + 9.0 * r * ts +
             4.0 * r * tb + 7.0 * r * nc + kPolyStride * r * nc;
  // flux: face cells and wall flag, Gauss data, polynomials read, face fluxes written
  bytes[1] = 9.0 * nf + 40.0 * r * nf + kPolyStride * r * nc + kFaceStride * r * nf;
  // face sums + stage update: CSR, face fluxes, 1/|Omega| (8 B), the state's gather copy read,
  // L and Lt (written by stage 1, read by stage 2, 8 B per value), the new gather copy written;
  // the FP64-update mode reads the FP64 state (40 B) in place of the gather copy and writes it
  // back in stage 2 (half of the passes: 20 B per pass on average)
  bytes[2] = 4.0 * (nc + 1) + 4.0 * ncf + kFaceStride * r * nf + 8.0 * nc +
             (s->fp64upd ? 60.0 : 48.0) * nc + 80.0 * nc + 48.0 * nc;
  return GKS_OK;
}

gks_status gks_launches_per_pass(const gks_solver* s, int64_t launches[3]) {
  if (!s || !launches) return GKS_E_INVAL;
  launches[0] = 0;
  for (int r = 0; r < s->m.rr.n; ++r) launches[0] += s->m.rr.t1[r] > s->m.rr.t0[r] ? 1 : 0;
  if (s->m.ng > 0) launches[0] += 1;  // the ghost refresh of moving no-slip walls
  launches[1] = 1;
  launches[2] = 1;
  return GKS_OK;
}

gks_status gks_timing_enable(gks_solver* s, int enable) {
  if (!s) return GKS_E_INVAL;
  s->timing = enable != 0;
  return GKS_OK;
}

gks_status gks_timing_read(gks_solver* s, double ms[3], int64_t counts[3]) {
  if (!s || !ms || !counts) return GKS_E_INVAL;
  cudaError_t e = cudaStreamSynchronize(s->st);
  if (e != cudaSuccess) return s->cuda_fail(e, "timing synchronise");
  for (int k = 0; k < 3; ++k) {
    ms[k] = 0.0;
    counts[k] = 0;
  }
  for (auto& u : s->ev_used) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, u.second.first, u.second.second) == cudaSuccess && u.first < 3) {
      ms[u.first] += t;
      counts[u.first] += 1;
    }
    s->ev_pool.push_back(u.second.first);
    s->ev_pool.push_back(u.second.second);
  }
  s->ev_used.clear();
  return GKS_OK;
}

const char* gks_last_error(const gks_solver* s) {
  return s ? s->err.c_str() : g_mesh_err.c_str();
}

void gks_destroy(gks_solver* s) {
  if (!s) return;
  if (s->st) cudaStreamSynchronize(s->st);
  else cudaDeviceSynchronize();
  for (void* p : s->owned) cudaFree(p);
  for (auto& u : s->ev_used) {
    cudaEventDestroy(u.second.first);
    cudaEventDestroy(u.second.second);
  }
  for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
  for (int k = 0; k < s->fj.n; ++k) {
    cudaStreamSynchronize(s->fj.aux[k]);
    cudaStreamDestroy(s->fj.aux[k]);
    cudaEventDestroy(s->fj.join[k]);
  }
  if (s->fj.fork) cudaEventDestroy(s->fj.fork);
  if (s->h_dt) cudaFreeHost(s->h_dt);
  delete s;
}

}  // extern "C"

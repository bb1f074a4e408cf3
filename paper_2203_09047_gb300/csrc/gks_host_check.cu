// Host instantiations of the Gauss-point flux and its vector-Jacobian product in FP64, running
// the same templated arithmetic as the flux kernels. They let the kinetic formulas and their
// hand-written adjoint be checked on a CPU (against the oracle and finite differences). One
// device entry runs the FP32 Gauss-point flux in its scalar and its packed f32x2 instantiation
// side by side, a direct test of the pair arithmetic.
#include <cstdint>

#include <cuda_runtime.h>

#include "gks_flux_f32x2.cuh"
#include "gks_kinetic_adj.cuh"

namespace {
gks::FluxParams<double> params_from(const double* p) {
  // p = {gamma, mu, tau_eps, tau_C, flux_mode, tau_model, Pr, T_ref, mu_pow,
  //      wall_u[6][3], wall_T[6], farfield[6][5]}
  gks::FluxParams<double> P;
  P.gamma = p[0];
  P.K = (5.0 - 3.0 * p[0]) / (p[0] - 1.0);
  P.mu = p[1];
  P.tau_eps = p[2];
  P.tau_C = p[3];
  P.full = (int)p[4];
  P.tau_model = (int)p[5];
  P.pr_fix = 1.0 / p[6] - 1.0;
  P.T_ref = p[7];
  P.mu_pow = p[8];
  return P;
}
// the wall plane of `code` from p's wall_u[6][3], wall_T[6]
gks::WallData<double> wall_from(const double* p, int code) {
  gks::WallData<double> d;
  if (code >= 6) {
    const int w = code % 6;
    for (int a = 0; a < 3; ++a) d.uw[a] = p[9 + 3 * w + a];
    d.Tw = p[27 + w];
    d.finf = p + 33 + 5 * w;  // the caller's vector holds the plane's far-field state
  }
  return d;
}
}  // namespace

// Local-frame Gauss-point flux: Fn = F^n, Ft = dF/dt (0 on success, 1 for a non-physical state).
extern "C" int gks_gp_flux_host(const double* p, const double* ql, const double* dql,
                                const double* qr, const double* dqr, double dt, double* Fn,
                                double* Ft) {
  const gks::FluxParams<double> P = params_from(p);
  double a[3][5], b[3][5];
  for (int d = 0; d < 3; ++d)
    for (int v = 0; v < 5; ++v) {
      a[d][v] = dql[5 * d + v];
      b[d][v] = dqr[5 * d + v];
    }
  return gks::gks_gp_flux(P, ql, a, qr, b, dt, Fn, Ft) ? 0 : 1;
}

// Its vector-Jacobian product: cotangents (gFn, gFt) -> (gql, gdql[3][5], gqr, gdqr[3][5]).
extern "C" int gks_gp_flux_vjp_host(const double* p, const double* ql, const double* dql,
                                    const double* qr, const double* dqr, double dt,
                                    const double* gFn, const double* gFt, double* gql,
                                    double* gdql, double* gqr, double* gdqr) {
  const gks::FluxParams<double> P = params_from(p);
  double a[3][5], b[3][5], ga[3][5], gb[3][5];
  for (int d = 0; d < 3; ++d)
    for (int v = 0; v < 5; ++v) {
      a[d][v] = dql[5 * d + v];
      b[d][v] = dqr[5 * d + v];
      ga[d][v] = gb[d][v] = 0.0;
    }
  for (int v = 0; v < 5; ++v) gql[v] = gqr[v] = 0.0;
  if (!gks::gks_gp_flux_vjp_cf(P, ql, a, qr, b, dt, gFn, gFt, gql, ga, gqr, gb)) return 1;
  for (int d = 0; d < 3; ++d)
    for (int v = 0; v < 5; ++v) {
      gdql[5 * d + v] = ga[d][v];
      gdqr[5 * d + v] = gb[d][v];
    }
  return 0;
}

// Global-frame Gauss-point contribution (values, gradients [5][3], unit normal, weight) and its
// vector-Jacobian product; gacc = nullptr runs the forward only (acc[10]).
extern "C" int gks_gp_face_host(const double* p, const double* vl, const double* gl,
                                const double* vr, const double* gr, const double* n1, double w,
                                double dt, double* acc, const double* gacc, double* gvl,
                                double* ggl, double* gvr, double* ggr) {
  const gks::FluxParams<double> P = params_from(p);
  double GL[5][3], GR[5][3];
  for (int v = 0; v < 5; ++v)
    for (int a = 0; a < 3; ++a) {
      GL[v][a] = gl[3 * v + a];
      GR[v][a] = gr[3 * v + a];
    }
  if (!gks::gp_flux_global(P, vl, GL, vr, GR, n1, w, dt, acc)) return 1;
  if (!gacc) return 0;
  double gGL[5][3] = {}, gGR[5][3] = {};
  for (int v = 0; v < 5; ++v) gvl[v] = gvr[v] = 0.0;
  if (!gks::gp_flux_global_vjp(P, vl, GL, vr, GR, n1, w, dt, gacc, gvl, gGL, gvr, gGR)) return 1;
  for (int v = 0; v < 5; ++v)
    for (int a = 0; a < 3; ++a) {
      ggl[3 * v + a] = gGL[v][a];
      ggr[3 * v + a] = gGR[v][a];
    }
  return 0;
}

// The wall ghost at a Gauss point (value, gradient [5][3]) for wall code `code`, and, when gvg is
// given, the reverse pass: (gvg, ggg) -> (gv, gg) (overwritten).
extern "C" void gks_wall_ghost_host(const double* p, int code, const double* v, const double* g,
                                    double* vg, double* gg, const double* gvg, const double* ggg,
                                    double* gv, double* gga) {
  const gks::FluxParams<double> P = params_from(p);
  double G[5][3], GG[5][3];
  for (int r = 0; r < 5; ++r)
    for (int b = 0; b < 3; ++b) G[r][b] = g[3 * r + b];
  const gks::WallData<double> wd = wall_from(p, code);
  gks::wall_ghost(P, code, wd, v, G, vg, GG);
  for (int r = 0; r < 5; ++r)
    for (int b = 0; b < 3; ++b) gg[3 * r + b] = GG[r][b];
  if (!gvg) return;
  double Y[5][3], A[5][3] = {};
  for (int r = 0; r < 5; ++r) {
    gv[r] = 0.0;
    for (int b = 0; b < 3; ++b) Y[r][b] = ggg[3 * r + b];
  }
  if (code >= 12)  // far field: a function of the owner's value only
    gks::farfield_state_vjp(P, wd.finf, code % 3, (code % 6) >= 3 ? 1.0 : -1.0, v, gvg, gv);
  else
    gks::wall_ghost_vjp(P, code, wd, v, G, gvg, Y, gv, A);
  for (int r = 0; r < 5; ++r)
    for (int b = 0; b < 3; ++b) gga[3 * r + b] = A[r][b];
}

// The wall treatment of a face's summed flux acc[10] (in place).
extern "C" void gks_wall_flux_fix_host(const double* p, int code, double* acc) {
  gks::wall_flux_fix(code, wall_from(p, code), acc);
}

namespace {
gks::FluxParams<float> params_f32(const double* p) {
  const gks::FluxParams<double> d = params_from(p);
  gks::FluxParams<float> P;
  P.gamma = (float)d.gamma;
  P.K = (float)d.K;
  P.mu = (float)d.mu;
  P.tau_eps = (float)d.tau_eps;
  P.tau_C = (float)d.tau_C;
  P.full = d.full;
  P.tau_model = d.tau_model;
  P.pr_fix = (float)d.pr_fix;
  P.T_ref = (float)d.T_ref;
  P.mu_pow = (float)d.mu_pow;
  return P;
}
// point i: in[45 i ..] = vl[5], gl[5][3], vr[5], gr[5][3], n1[3], w, dt;
// out[21 i ..] = scalar acc[10], packed acc[10], (scalar ok) + 2 (packed ok)
__global__ void k_face_f32_pair(gks::FluxParams<float> P, int n, const float* __restrict__ in,
                                float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float* x = in + 45 * (int64_t)i;
  float vl[5], gl[5][3], vr[5], gr[5][3], n1[3];
  for (int v = 0; v < 5; ++v) {
    vl[v] = x[v];
    vr[v] = x[20 + v];
    for (int a = 0; a < 3; ++a) {
      gl[v][a] = x[5 + 3 * v + a];
      gr[v][a] = x[25 + 3 * v + a];
    }
  }
  for (int a = 0; a < 3; ++a) n1[a] = x[40 + a];
  const float w = x[43], dt = x[44];
  float acc_s[10], acc_p[10];
  const bool ok_s = gks::gp_flux_global(P, vl, gl, vr, gr, n1, w, dt, acc_s);
  const bool ok_p = gks::gp_flux_global2(P, vl, gl, vr, gr, n1, w, dt, acc_p);
  float* o = out + 21 * (int64_t)i;
  for (int q = 0; q < 10; ++q) {
    o[q] = acc_s[q];
    o[10 + q] = acc_p[q];
  }
  o[20] = (ok_s ? 1.f : 0.f) + (ok_p ? 2.f : 0.f);
}
}  // namespace

// The FP32 Gauss-point contribution on the GPU in the scalar and the packed f32x2
// instantiation of the flux templates, for n points: in [n][45], out [n][21] (device
// pointers, layout above), p the parameter vector of gks_gp_face_host. Synchronises the
// device; 0 on success, 1 on a CUDA error.
extern "C" int gks_gp_face_f32_pair(const double* p, int n, const float* in, float* out) {
  if (n <= 0) return 0;
  k_face_f32_pair<<<(n + 127) / 128, 128>>>(params_f32(p), n, in, out);
  return cudaDeviceSynchronize() == cudaSuccess ? 0 : 1;
}


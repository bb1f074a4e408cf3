// Vector-Jacobian product of the residual (L, Lt)(Q) for a fixed dt, in FP64:
//   gQ = (dL/dQ)^T gL + (dLt/dQ)^T gLt.
// The forward reconstruction polynomials are recomputed by the forward kernel; the adjoint runs
// in four deterministic, atomic-free passes:
//   k_vjp_flux     per face Gauss point: face cotangent from gL, gLt of the two cells, reverse of
//                  the gas-kinetic flux and of the polynomial evaluation; per-face write of the
//                  cotangents of both sides' polynomial coefficients
//   k_vjp_poly     per cell: sum of its faces' polynomial cotangents (fixed face order)
//   k_vjp_recon    per cell: reverse of the WENO reconstruction (combination, nonlinear weights,
//                  smoothness indicators, least squares) -> cotangents of every stencil difference
//   k_vjp_stencil  per cell: sum over the reverse stencil (the entries that reference the cell)
#include <cuda_runtime.h>

#include "gks_device.cuh"
#include "gks_kinetic_adj.cuh"

namespace gks {
namespace {

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

struct PolyRef64 {
  const double* __restrict__ p;
  __device__ __forceinline__ double operator()(int v, int j) const { return p[10 * v + j]; }
};

// Positivity fallback (the forward flux's, mirrored): a side whose reconstructed Gauss-point
// state has rho <= 0 or p <= 0 takes its cell average with a zero gradient. Here the cell average
// is written as the mean of the cell's own polynomial, c0 + sum_j c_j <d_j> over the quadratic
// terms (<d_j> the cell's central second moments: scaled moments times h^2), which equals the
// cell average for every state, so that its cotangent flows back through the reconstruction.
__device__ __forceinline__ bool nonphysical(const double v[5]) {
  const double m2 = v[1] * v[1] + v[2] * v[2] + v[3] * v[3];
  return !(v[0] > 0.0 && v[0] * v[4] > 0.5 * m2);
}
__device__ __forceinline__ void central_moments(const double* __restrict__ mom,
                                                const double* __restrict__ hcell, int64_t nc,
                                                int64_t c, double mu[6]) {
  const double h2 = hcell[c] * hcell[c];
#pragma unroll
  for (int q = 0; q < 6; ++q) mu[q] = mom[q * nc + c] * h2;
}
__device__ __forceinline__ void poly_mean(const double* __restrict__ p, const double mu[6],
                                          double v[5], double g[5][3]) {
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    double s = p[10 * k];
#pragma unroll
    for (int q = 0; q < 6; ++q) s += p[10 * k + 4 + q] * mu[q];
    v[k] = s;
#pragma unroll
    for (int a = 0; a < 3; ++a) g[k][a] = 0.0;
  }
}
__device__ __forceinline__ void poly_mean_adj(const double mu[6], const double gv[5],
                                              double gp[5][10]) {
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    gp[k][0] += gv[k];
#pragma unroll
    for (int q = 0; q < 6; ++q) gp[k][4 + q] += gv[k] * mu[q];
  }
}

// kFull and kTau0 fix the flux form and a zero collision time at compile time (as in the forward
// kernel), so that each instance holds only its own form's recomputed forward state. kWalls =
// false is the instance for meshes without boundary planes (every face has two cells; no
// boundary code compiled in), true the one that handles both kinds of face.
template <bool kFull, bool kTau0, bool kWalls>
__global__ void __launch_bounds__(128) k_vjp_flux(
    int64_t nf, const int32_t* __restrict__ f_owner, const int32_t* __restrict__ f_nb,
    const int8_t* __restrict__ f_wall, const double* __restrict__ fgp,
    const double* __restrict__ poly, const double* __restrict__ gL, const double* __restrict__ gLt,
    const double* __restrict__ vol, int64_t nc, FluxParams<double> P,
    const double* __restrict__ wall_tab, double dt, int fallback, const double* __restrict__ mom,
    const double* __restrict__ hcell, double* __restrict__ gpf, int* flag) {
  P.full = kFull;
  if (kTau0) P.tau_model = 0;
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t f = gid >> 2;
  const bool active = f < nf;
  double go[5][10], gn[5][10];
#pragma unroll
  for (int v = 0; v < 5; ++v)
#pragma unroll
    for (int j = 0; j < 10; ++j) go[v][j] = gn[v][j] = 0.0;
  if (active) {
    const int64_t stride = 4 * nf;
    const int32_t o = f_owner[f], nb = f_nb[f];
    const int wall = f_wall[f];
    // cotangent of the face flux: L_o -= F / |O_o|, L_nb += F / |O_nb|
    double gacc[10];
    const double io = 1.0 / vol[o];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      gacc[q] = -gL[q * nc + o] * io;
      gacc[5 + q] = -gLt[q * nc + o] * io;
    }
    if (!kWalls || nb >= 0) {
      const double in = 1.0 / vol[nb];
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        gacc[q] += gL[q * nc + nb] * in;
        gacc[5 + q] += gLt[q * nc + nb] * in;
      }
    } else {
      wall_flux_fix_adj(wall, wall_data(wall_tab, wall), gacc);  // the wall treatment, reversed
    }
    double dl[3], dr[3], n1[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      dl[a] = fgp[a * stride + gid];
      dr[a] = fgp[(3 + a) * stride + gid];
      n1[a] = fgp[(6 + a) * stride + gid];
    }
    const double w = fgp[9 * stride + gid];
    double vl[5], gl[5][3], vr[5], gr[5][3];
    eval_poly(PolyRef64{poly + (int64_t)kPolyStride * o}, dl, vl, gl);
    const bool fbl = fallback && nonphysical(vl);
    double mu[6];
    if (fbl) {
      central_moments(mom, hcell, nc, o, mu);
      poly_mean(poly + (int64_t)kPolyStride * o, mu, vl, gl);
    }
    bool fbr = false;
    if (!kWalls || nb >= 0) {
      eval_poly(PolyRef64{poly + (int64_t)kPolyStride * nb}, dr, vr, gr);
      fbr = fallback && nonphysical(vr);
      if (fbr) {
        double mun[6];
        central_moments(mom, hcell, nc, nb, mun);
        poly_mean(poly + (int64_t)kPolyStride * nb, mun, vr, gr);
      }
    } else {
      wall_ghost<double, true>(P, wall, wall_data(wall_tab, wall), vl, gl, vr, gr);
    }
    double gvl[5] = {0, 0, 0, 0, 0}, gvr[5] = {0, 0, 0, 0, 0};
    double ggl[5][3], ggr[5][3];
#pragma unroll
    for (int v = 0; v < 5; ++v)
#pragma unroll
      for (int a = 0; a < 3; ++a) ggl[v][a] = ggr[v][a] = 0.0;
    if (gp_flux_global_vjp(P, vl, gl, vr, gr, n1, w, dt, gacc, gvl, ggl, gvr, ggr)) {
      // the wall's ghost is a function of the owner's value and gradient: fold its cotangent back
      if (kWalls && nb < 0)
        wall_ghost_vjp(P, wall, wall_data(wall_tab, wall), vl, gl, gvr, ggr, gvl, ggl);
      if (fbl)
        poly_mean_adj(mu, gvl, go);
      else
        eval_poly_adj(dl, gvl, ggl, go);
      if (fbr) {
        double mun[6];
        central_moments(mom, hcell, nc, nb, mun);
        poly_mean_adj(mun, gvr, gn);
      } else if (!kWalls || nb >= 0) {
        eval_poly_adj(dr, gvr, ggr, gn);
      }
    } else {
      atomicOr(flag, kErrNonphysical);
    }
  }
#pragma unroll
  for (int v = 0; v < 5; ++v)
#pragma unroll
    for (int j = 0; j < 10; ++j) {
      go[v][j] += __shfl_xor_sync(0xffffffffu, go[v][j], 1);
      go[v][j] += __shfl_xor_sync(0xffffffffu, go[v][j], 2);
      gn[v][j] += __shfl_xor_sync(0xffffffffu, gn[v][j], 1);
      gn[v][j] += __shfl_xor_sync(0xffffffffu, gn[v][j], 2);
    }
  if (active && (gid & 3) == 0) {
    double* po = gpf + (int64_t)2 * kPolyStride * f;
    double* pn = po + kPolyStride;
#pragma unroll
    for (int v = 0; v < 5; ++v)
#pragma unroll
      for (int j = 0; j < 10; ++j) {
        po[10 * v + j] = go[v][j];
        pn[10 * v + j] = gn[v][j];
      }
  }
}

__global__ void k_vjp_poly(int64_t nc, const int32_t* __restrict__ cf_ptr,
                           const int32_t* __restrict__ cf_idx, const double* __restrict__ gpf,
                           double* __restrict__ gpc) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nc) return;
  double s[50];
#pragma unroll
  for (int q = 0; q < 50; ++q) s[q] = 0.0;
  for (int k = cf_ptr[i]; k < cf_ptr[i + 1]; ++k) {
    const int32_t e = cf_idx[k];
    const double* p = gpf + (int64_t)kPolyStride * (2 * (int64_t)(e >> 1) + (e & 1));
#pragma unroll
    for (int q = 0; q < 50; ++q) s[q] += p[q];
  }
  double* o = gpc + (int64_t)kPolyStride * i;
#pragma unroll
  for (int q = 0; q < 50; ++q) o[q] = s[q];
}

// Reverse of the reconstruction of one cell, one variable at a time (the variables are
// independent: each has its own weights).
__global__ void __launch_bounds__(64) k_vjp_recon(
    int64_t nc, const double* __restrict__ QA, const int32_t* __restrict__ t_K,
    const uint64_t* __restrict__ t_cnt, const int32_t* __restrict__ t_st,
    const int32_t* __restrict__ t_sb, const int32_t* __restrict__ t_idx,
    const int32_t* __restrict__ st_ptr, const int8_t* __restrict__ n_sub,
    const double* __restrict__ Ap, const double* __restrict__ Bp, const double* __restrict__ mom,
    const double* __restrict__ hcell, double wg, double weps, int wpow,
    const double* __restrict__ gpc, double* __restrict__ gdq, double* __restrict__ gq0) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nc) return;
  const int64_t tile = i / kTile;
  const int lane = (int)(i % kTile);
  const int K = st_ptr[i + 1] - st_ptr[i];  // the cell's own members (tile padding excluded)
  const int KT = t_K[tile];
  const uint64_t cnt = t_cnt[tile];
  const int M = n_sub[i];
  const int64_t row0 = t_st[tile];
  const int32_t* sidx = t_idx + row0 * kTile + lane;
  const double* A = Ap + row0 * 9 * kTile + lane;
  const double* Bt = Bp + ((int64_t)t_sb[tile] * kTile + lane) * 4;  // [slot][lane][4]
  double* gdqc = gdq + row0 * 5 * kTile + lane;
  double m2[6];
  for (int q = 0; q < 6; ++q) m2[q] = mom[q * nc + i];
  const double h = hcell[i], ih = 1.0 / h, ih2 = ih * ih;
  const double g0 = 1.0 - wg * M;
  double c0q[5];
  for (int v = 0; v < 5; ++v) c0q[v] = QA[6 * i + v];
  for (int v = 0; v < 5; ++v) {
    // ---- forward: stencil differences, a, b_m, indicators, weights
    double dq[kMaxStencil];
    for (int k = 0; k < KT; ++k) {
      const int32_t e = sidx[k * kTile];
      double q = QA[6 * (int64_t)(e & kCellMask) + v];
      if (v >= 1 && v <= 3 && ((e >> (kFlipShift + v - 1)) & 1)) q = -q;
      dq[k] = q - c0q[v];
    }
    double a[9];
    for (int n = 0; n < 9; ++n) {
      double s = 0.0;
      for (int k = 0; k < KT; ++k) s += A[(9 * k + n) * kTile] * dq[k];
      a[n] = s;
    }
    double b[kMaxSub][3], bet[kMaxSub];
    {
      const double* e = Bt;
      for (int s = 0; s < kMaxSub; ++s) {
        const int cs = (int)((cnt >> (8 * s)) & 0xffu);
        b[s][0] = b[s][1] = b[s][2] = 0.0;
        for (int j = 0; j < cs; ++j, e += 4 * kTile) {
          const int k = (int)e[3];
          for (int t = 0; t < 3; ++t) b[s][t] += e[t] * dq[k];
        }
        bet[s] = b[s][0] * b[s][0] + b[s][1] * b[s][1] + b[s][2] * b[s][2];
      }
    }
    const double gx[3] = {2 * a[3], a[6], a[7]};
    const double gy[3] = {a[6], 2 * a[4], a[8]};
    const double gz[3] = {a[7], a[8], 2 * a[5]};
    auto mv = [&](const double g[3], double o[3]) {
      o[0] = m2[0] * g[0] + m2[3] * g[1] + m2[4] * g[2];
      o[1] = m2[3] * g[0] + m2[1] * g[1] + m2[5] * g[2];
      o[2] = m2[4] * g[0] + m2[5] * g[1] + m2[2] * g[2];
    };
    double hx[3], hy[3], hz[3];
    mv(gx, hx);
    mv(gy, hy);
    mv(gz, hz);
    const double beta0 = a[0] * a[0] + a[1] * a[1] + a[2] * a[2] +
                         (gx[0] * hx[0] + gx[1] * hx[1] + gx[2] * hx[2]) +
                         (gy[0] * hy[0] + gy[1] * hy[1] + gy[2] * hy[2]) +
                         (gz[0] * hz[0] + gz[1] * hz[1] + gz[2] * hz[2]) +
                         4 * (a[3] * a[3] + a[4] * a[4] + a[5] * a[5]) + a[6] * a[6] +
                         a[7] * a[7] + a[8] * a[8];
    double tau = 0.0;
    for (int s = 0; s < M; ++s) tau += fabs(beta0 - bet[s]);
    tau /= M;
    auto ratio_pow = [&](double r) {
      double p = r;
      for (int e = 1; e < wpow; ++e) p *= r;
      return p;
    };
    double w[kMaxSub + 1], rr[kMaxSub + 1];
    rr[0] = tau / (beta0 + weps);
    w[0] = g0 * (1.0 + ratio_pow(rr[0]));
    double S = w[0];
    for (int s = 0; s < M; ++s) {
      rr[s + 1] = tau / (bet[s] + weps);
      w[s + 1] = wg * (1.0 + ratio_pow(rr[s + 1]));
      S += w[s + 1];
    }
    const double wb0 = w[0] / S;
    const double ca = wb0 / g0;
    double cs[kMaxSub];
    for (int s = 0; s < M; ++s) cs[s] = w[s + 1] / S - wb0 * wg / g0;
    // ---- reverse
    const double* go = gpc + (int64_t)kPolyStride * i + 10 * v;
    double gQ0 = go[0];
    double gC[9];
    for (int n = 0; n < 3; ++n) gC[n] = go[1 + n] * ih;
    for (int n = 3; n < 9; ++n) gC[n] = go[1 + n] * ih2 - go[0] * m2[n - 3];
    double ga[9], gb[kMaxSub][3];
    double gca = 0.0;
    for (int n = 0; n < 9; ++n) {
      ga[n] = ca * gC[n];
      gca += gC[n] * a[n];
    }
    double gcs[kMaxSub];
    for (int s = 0; s < kMaxSub; ++s) {
      gb[s][0] = gb[s][1] = gb[s][2] = 0.0;
      gcs[s] = 0.0;
    }
    for (int s = 0; s < M; ++s)
      for (int t = 0; t < 3; ++t) {
        gb[s][t] = cs[s] * gC[t];
        gcs[s] += gC[t] * b[s][t];
      }
    // ca = wb0/g0, cs_s = wb_s - wb0 wg/g0
    double gwb[kMaxSub + 1];
    gwb[0] = gca / g0;
    for (int s = 0; s < M; ++s) {
      gwb[0] -= gcs[s] * wg / g0;
      gwb[s + 1] = gcs[s];
    }
    // wb_j = w_j / S
    double dotw = 0.0;
    for (int j = 0; j <= M; ++j) dotw += gwb[j] * (w[j] / S);
    double gtau = 0.0, gbeta0 = 0.0, gbet[kMaxSub];
    for (int s = 0; s < kMaxSub; ++s) gbet[s] = 0.0;
    for (int j = 0; j <= M; ++j) {
      const double gw = (gwb[j] - dotw) / S;
      const double gam = j == 0 ? g0 : wg;
      const double r = rr[j];
      double dpow = wpow;  // d(r^p)/dr = p r^(p-1)
      for (int e = 1; e < wpow; ++e) dpow *= r;
      const double gr = gw * gam * dpow;
      const double bb = j == 0 ? beta0 : bet[j - 1];
      gtau += gr / (bb + weps);
      const double gbb = -gr * tau / ((bb + weps) * (bb + weps));
      if (j == 0)
        gbeta0 += gbb;
      else
        gbet[j - 1] += gbb;
    }
    // tau = sum_s |beta0 - beta_s| / M  (derivative of |x| taken as +1 at x = 0)
    for (int s = 0; s < M; ++s) {
      const double sg = (beta0 - bet[s]) < 0.0 ? -1.0 : 1.0;
      gbeta0 += sg * gtau / M;
      gbet[s] -= sg * gtau / M;
    }
    // beta_s = |b_s|^2
    for (int s = 0; s < M; ++s)
      for (int t = 0; t < 3; ++t) gb[s][t] += 2.0 * b[s][t] * gbet[s];
    // beta0
    for (int n = 0; n < 3; ++n) ga[n] += 2.0 * a[n] * gbeta0;
    ga[3] += (2.0 * (2.0 * hx[0]) + 8.0 * a[3]) * gbeta0;
    ga[4] += (2.0 * (2.0 * hy[1]) + 8.0 * a[4]) * gbeta0;
    ga[5] += (2.0 * (2.0 * hz[2]) + 8.0 * a[5]) * gbeta0;
    ga[6] += (2.0 * hx[1] + 2.0 * hy[0] + 2.0 * a[6]) * gbeta0;
    ga[7] += (2.0 * hx[2] + 2.0 * hz[0] + 2.0 * a[7]) * gbeta0;
    ga[8] += (2.0 * hy[2] + 2.0 * hz[1] + 2.0 * a[8]) * gbeta0;
    // a = A+ dq, b_s = B_s dq|S_s
    double gd[kMaxStencil];
    for (int k = 0; k < KT; ++k) {
      double s = 0.0;
      for (int n = 0; n < 9; ++n) s += A[(9 * k + n) * kTile] * ga[n];
      gd[k] = s;
    }
    {
      const double* e = Bt;
      for (int s = 0; s < kMaxSub; ++s) {
        const int csn = (int)((cnt >> (8 * s)) & 0xffu);
        for (int j = 0; j < csn; ++j, e += 4 * kTile) {
          const int k = (int)e[3];
          for (int t = 0; t < 3; ++t) gd[k] += e[t] * gb[s][t];
        }
      }
    }
    for (int k = 0; k < KT; ++k) {
      gQ0 -= gd[k];
      gdqc[(5 * k + v) * kTile] = k < K ? gd[k] : 0.0;
    }
    gq0[v * nc + i] = gQ0;
  }
}

// One boundary plane's map of a ghost cell's flow variables (as k_ghost_fill applies it):
// slip, normal momentum negated; no-slip with velocity t[0..2], m -> 2 U_w rho - m,
// E -> E + 2 |U_w|^2 rho - 2 U_w . m; far field, the characteristic state. And its
// transposed Jacobian at q applied to y, added to g.
__device__ void plane_map(const FluxParams<double>& P, int w, int kind, const double* t,
                          const double q[5], double out[5]) {
  const int ax = w % 3;
  if (kind == 3) {
    farfield_state(P, t + 4, ax, w >= 3 ? 1.0 : -1.0, q, out);
    return;
  }
  for (int v = 0; v < 5; ++v) out[v] = q[v];
  if (kind == 1) {
    out[1 + ax] = -q[1 + ax];
    return;
  }
  const double um = t[0] * q[1] + t[1] * q[2] + t[2] * q[3];
  out[4] = q[4] + 2.0 * (t[0] * t[0] + t[1] * t[1] + t[2] * t[2]) * q[0] - 2.0 * um;
  for (int a = 0; a < 3; ++a) out[1 + a] = 2.0 * t[a] * q[0] - q[1 + a];
}
__device__ void plane_map_vjp(const FluxParams<double>& P, int w, int kind, const double* t,
                              const double q[5], const double y[5], double g[5]) {
  const int ax = w % 3;
  if (kind == 3) {
    farfield_state_vjp(P, t + 4, ax, w >= 3 ? 1.0 : -1.0, q, y, g);
    return;
  }
  if (kind == 1) {
    for (int v = 0; v < 5; ++v) g[v] += (v == 1 + ax) ? -y[v] : y[v];
    return;
  }
  const double uw2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
  g[0] += y[0] + 2.0 * (t[0] * y[1] + t[1] * y[2] + t[2] * y[3]) + 2.0 * uw2 * y[4];
  for (int a = 0; a < 3; ++a) g[1 + a] += -y[1 + a] - 2.0 * t[a] * y[4];
  g[4] += y[4];
}

__global__ void k_vjp_stencil(int64_t nc, const int32_t* __restrict__ rs_ptr,
                              const int32_t* __restrict__ rs_pos, const int32_t* __restrict__ t_idx,
                              const double* __restrict__ g_map, const uint8_t* __restrict__ g_chain,
                              int bcs, FluxParams<double> P, const double* __restrict__ wall_tab,
                              const double* __restrict__ QA, const double* __restrict__ gdq,
                              const double* __restrict__ gq0, double* __restrict__ gQ) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= nc) return;
  double s[5];
  for (int v = 0; v < 5; ++v) s[v] = gq0[v * nc + j];
  for (int k = rs_ptr[j]; k < rs_ptr[j + 1]; ++k) {
    const int64_t pos = rs_pos[k];
    const int32_t e = t_idx[pos];
    const int fl = e >> kFlipShift;
    const int64_t slot = pos / kTile, lane = pos % kTile;
    const double* g = gdq + slot * 5 * kTile + lane;
    double y[5];
    for (int v = 0; v < 5; ++v) y[v] = g[v * kTile];
    if ((e & kCellMask) >= nc && g_chain[(e & kCellMask) - nc]) {
      // a ghost slot across a far-field plane: the planes' maps reversed at this cell's state
      const int code = g_chain[(e & kCellMask) - nc];
      const int w0 = (code & 7) - 1, w1 = ((code >> 3) & 7) - 1;
      double q0[5], q1[5], y0[5] = {0, 0, 0, 0, 0};
      for (int v = 0; v < 5; ++v) q0[v] = QA[6 * j + v];
      const int k0 = (bcs >> (2 * (w0 % 3))) & 3;
      if (w1 >= 0) {
        const int k1 = (bcs >> (2 * (w1 % 3))) & 3;
        plane_map(P, w0, k0, wall_tab + kPlaneStride * w0, q0, q1);
        plane_map_vjp(P, w1, k1, wall_tab + kPlaneStride * w1, q1, y, y0);
      } else {
        for (int v = 0; v < 5; ++v) y0[v] = y[v];
      }
      plane_map_vjp(P, w0, k0, wall_tab + kPlaneStride * w0, q0, y0, s);
      continue;
    }
    if ((e & kCellMask) >= nc) {
      // a wall ghost slot: the transpose of its map (rho, m_j, E) -> (rho, s_j m_j + a_j rho,
      // E + b rho + c . m)
      const double* c = g_map + 10 * ((e & kCellMask) - nc);
      s[0] += y[0] + c[3] * y[1] + c[4] * y[2] + c[5] * y[3] + c[6] * y[4];
      for (int a = 0; a < 3; ++a) s[1 + a] += c[a] * y[1 + a] + c[7 + a] * y[4];
      s[4] += y[4];
      continue;
    }
    for (int v = 0; v < 5; ++v) {
      double x = y[v];
      if (v >= 1 && v <= 3 && ((fl >> (v - 1)) & 1)) x = -x;
      s[v] += x;
    }
  }
  for (int v = 0; v < 5; ++v) gQ[v * nc + j] = s[v];
}

}  // namespace

void launch_vjp(const DevMesh& m, const Geo64& g64, const GeoR<double>& g, const KParams<double>& p,
                const double* QA, const double* poly, const double* gL, const double* gLt,
                double dt, double* gpf, double* gpc, double* gdq, double* gq0, double* gQ,
                const int32_t* rs_ptr, const int32_t* rs_pos, int* flag, cudaStream_t st) {
  const FluxParams<double> fp = flux_params(p);
  using Kern = decltype(&k_vjp_flux<true, true, true>);
  const Kern tab[2][2][2] = {
      {{k_vjp_flux<false, false, false>, k_vjp_flux<false, false, true>},
       {k_vjp_flux<false, true, false>, k_vjp_flux<false, true, true>}},
      {{k_vjp_flux<true, false, false>, k_vjp_flux<true, false, true>},
       {k_vjp_flux<true, true, false>, k_vjp_flux<true, true, true>}}};
  const Kern kern = tab[fp.full ? 1 : 0][fp.tau_model == 0 ? 1 : 0][m.bcs != 0 ? 1 : 0];
  // the flux adjoint keeps kilobytes of spilled state per thread in its stack frame (4-6 KB for
  // the full flux): raise the context's per-thread stack limit to cover it before the launch
  cudaFuncAttributes at;
  size_t cur = 0;
  if (cudaFuncGetAttributes(&at, kern) == cudaSuccess &&
      cudaDeviceGetLimit(&cur, cudaLimitStackSize) == cudaSuccess && at.localSizeBytes > cur)
    cudaDeviceSetLimit(cudaLimitStackSize, at.localSizeBytes);
  kern<<<blocks_for(4 * m.nf, 128), 128, 0, st>>>(m.nf, m.f_owner, m.f_nb, m.f_wall, g.fgp, poly,
                                                  gL, gLt, g64.vol, m.nc, fp, m.wall64, dt,
                                                  p.gp_fallback, g.mom, g.h, gpf, flag);
  k_vjp_poly<<<blocks_for(m.nc, 128), 128, 0, st>>>(m.nc, m.cf_ptr, m.cf_idx, gpf, gpc);
  k_vjp_recon<<<blocks_for(m.nc, 64), 64, 0, st>>>(m.nc, QA, m.t_K, m.t_cnt, m.t_st, m.t_sb,
                                                     m.t_idx, m.st_ptr, m.n_sub, g.Ap, g.Bp, g.mom,
                                                     g.h, p.weno_gamma, p.weno_eps, p.weno_pow, gpc,
                                                     gdq, gq0);
  k_vjp_stencil<<<blocks_for(m.nc, 128), 128, 0, st>>>(m.nc, rs_ptr, rs_pos, m.t_idx, m.g_map,
                                                        m.g_chain, m.bcs, fp, m.wall64, QA,
                                                        gdq, gq0, gQ);
}

}  // namespace gks

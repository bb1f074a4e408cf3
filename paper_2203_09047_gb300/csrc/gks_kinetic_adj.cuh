// Reverse-mode (vector-Jacobian) companion of gks_kinetic.cuh: the boundary treatment, the frame
// rotation and the polynomial evaluation around the Gauss-point flux, reversed by hand in the
// reverse order of the forward code; the flux itself is reversed in gks_kinetic_rev.cuh.
// Forward intermediates are recomputed (no tape).
#pragma once

#include "gks_kinetic.cuh"
#include "gks_kinetic_rev.cuh"

namespace gks {

// Reverse of wall_flux_fix: the cotangent of the treated face flux -> that of the summed one.
template <class R>
GKS_HD void wall_flux_fix_adj(int code, const WallData<R>& wd, R gacc[10]) {
  if (code >= 12) return;  // far field: the flux passes unchanged
  gacc[0] = gacc[5] = R(0);
  const int ax = code % 3;
  if (code < 6) {
#pragma unroll
    for (int v = 1; v < 5; ++v)
      if (v != 1 + ax) gacc[v] = gacc[5 + v] = R(0);
    return;
  }
  if (wd.Tw <= R(0)) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      gacc[1 + a] += wd.uw[a] * gacc[4];
      gacc[6 + a] += wd.uw[a] * gacc[9];
    }
    gacc[4] = gacc[9] = R(0);
  }
}

// Reverse of farfield_state: the cotangent y of the boundary state (conserved) -> that of the
// inside state q, added to g. Supersonic outflow passes y, supersonic inflow nothing; the
// subsonic state depends on q through R+ = u_n + 2c/(gamma-1) and, at an outflow, through the
// entropy p/rho^gamma and the tangential velocity.
template <class R>
GKS_HD void farfield_state_vjp(const FluxParams<R>& P, const R finf[5], int ax, R sg,
                               const R q[5], const R y[5], R g[5]) {
  const R gam = P.gamma, gm1 = P.gamma - R(1);
  const R ir = R(1) / q[0];
  const R U[3] = {q[1] * ir, q[2] * ir, q[3] * ir};
  const R U2 = U[0] * U[0] + U[1] * U[1] + U[2] * U[2];
  const R p = gm1 * (q[4] - R(0.5) * q[0] * U2);
  const R c = k_sqrt(gam * p * ir);
  const R un = sg * U[ax];
  if (un >= c) {
#pragma unroll
    for (int v = 0; v < 5; ++v) g[v] += y[v];
    return;
  }
  if (un <= -c) return;
  const R rinf = finf[0], pinf = finf[4];
  const R uninf = sg * finf[1 + ax];
  const R cinf = k_sqrt(gam * pinf / rinf);
  const R Rp = un + R(2) * c / gm1, Rm = uninf - R(2) * cinf / gm1;
  const R unb = R(0.5) * (Rp + Rm), cb = R(0.25) * gm1 * (Rp - Rm);
  const bool out_flow = unb >= R(0);
  const R s = out_flow ? p / k_pow(q[0], gam) : pinf / k_pow(rinf, gam);
  R Ub[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) Ub[a] = out_flow ? U[a] : finf[1 + a];
  Ub[ax] = sg * unb;
  const R rb = k_pow(cb * cb / (gam * s), R(1) / gm1);
  // out = (rb, rb Ub, pb/(gamma-1) + rb |Ub|^2 / 2), pb = rb cb^2 / gamma
  const R Ub2 = Ub[0] * Ub[0] + Ub[1] * Ub[1] + Ub[2] * Ub[2];
  R grb = y[0] + y[1] * Ub[0] + y[2] * Ub[1] + y[3] * Ub[2] + R(0.5) * Ub2 * y[4];
  R gUb[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) gUb[a] = rb * (y[1 + a] + y[4] * Ub[a]);
  const R gpb = y[4] / gm1;
  grb += gpb * cb * cb / gam;
  R gcb = gpb * R(2) * rb * cb / gam;
  // rb = (cb^2 / (gamma s))^(1/(gamma-1))
  gcb += grb * rb * R(2) / (gm1 * cb);
  const R gs = -grb * rb / (gm1 * s);
  const R gunb = sg * gUb[ax];
  const R gRp = R(0.5) * gunb + R(0.25) * gm1 * gcb;
  // back to the inside primitives
  R gU[3] = {R(0), R(0), R(0)}, grho = R(0), gp = R(0);
  if (out_flow) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
      if (a != ax) gU[a] += gUb[a];
    const R rg = k_pow(q[0], gam);
    gp += gs / rg;
    grho += -gs * gam * p / (rg * q[0]);
  }
  gU[ax] += sg * gRp;                      // R+ through u_n
  const R gc = gRp * R(2) / gm1;           // ... and through c = sqrt(gamma p / rho)
  gp += gc * c / (R(2) * p);
  grho += -gc * c / (R(2) * q[0]);
  // primitives -> conserved
  g[0] += grho - (gU[0] * U[0] + gU[1] * U[1] + gU[2] * U[2]) * ir + gp * gm1 * R(0.5) * U2;
#pragma unroll
  for (int a = 0; a < 3; ++a) g[1 + a] += gU[a] * ir - gp * gm1 * U[a];
  g[4] += gp * gm1;
}

// Reverse of wall_ghost: the cotangents (gvg, ggg) of the ghost value and gradient are added to
// those (gv, gg) of the owner's. The slip and adiabatic maps are linear (the transposed Jacobian
// and mirror); the isothermal map's energy row depends on U = m / rho also through the
// gradient's Jacobian, which adds the second-order term.
template <class R>
GKS_HD void wall_ghost_vjp(const FluxParams<R>& P, int code, const WallData<R>& wd, const R v[5],
                           const R g[5][3], const R gvg[5], const R ggg[5][3], R gv[5],
                           R gg[5][3]) {
  const int ax = code % 3;
  // far-field planes: the ghost is farfield_state of the owner's value only, with no gradient
  if (code >= 12) {
    farfield_state_vjp(P, wd.finf, ax, (code % 6) >= 3 ? R(1) : R(-1), v, gvg, gv);
    return;
  }
  if (code < 6) {
#pragma unroll
    for (int r = 0; r < 5; ++r) {
      const R sv = (r == 1 + ax) ? R(-1) : R(1);
      gv[r] += sv * gvg[r];
#pragma unroll
      for (int b = 0; b < 3; ++b) gg[r][b] += (b == ax ? -sv : sv) * ggg[r][b];
    }
    return;
  }
  const R uw[3] = {wd.uw[0], wd.uw[1], wd.uw[2]};
  const R uw2 = uw[0] * uw[0] + uw[1] * uw[1] + uw[2] * uw[2];
  const bool iso = wd.Tw > R(0);
  R j0, jm[3], j4, U[3] = {R(0), R(0), R(0)}, U2 = R(0), ir = R(0);
  if (iso) {
    ir = R(1) / v[0];
#pragma unroll
    for (int a = 0; a < 3; ++a) U[a] = v[1 + a] * ir;
    U2 = U[0] * U[0] + U[1] * U[1] + U[2] * U[2];
    j0 = R(2) * wd.Tw / (P.gamma - R(1)) - U2 + R(2) * uw2;
#pragma unroll
    for (int a = 0; a < 3; ++a) jm[a] = R(2) * (U[a] - uw[a]);
    j4 = R(-1);
  } else {
    j0 = R(2) * uw2;
#pragma unroll
    for (int a = 0; a < 3; ++a) jm[a] = R(-2) * uw[a];
    j4 = R(1);
  }
  // value: the Jacobian rows (1, 0..), (2 uw_a, -e_a, 0), (j0, jm, j4)
  gv[0] += gvg[0] + R(2) * (uw[0] * gvg[1] + uw[1] * gvg[2] + uw[2] * gvg[3]) + j0 * gvg[4];
#pragma unroll
  for (int a = 0; a < 3; ++a) gv[1 + a] += -gvg[1 + a] + jm[a] * gvg[4];
  gv[4] += j4 * gvg[4];
  // gradient: the same Jacobian after the mirror sign of each direction
  R D0 = R(0), Dm[3] = {R(0), R(0), R(0)};
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const R sb = b == ax ? R(-1) : R(1);
    const R z0 = sb * ggg[0][b], z4 = sb * ggg[4][b];
    R zm[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) zm[a] = sb * ggg[1 + a][b];
    gg[0][b] += z0 + R(2) * (uw[0] * zm[0] + uw[1] * zm[1] + uw[2] * zm[2]) + j0 * z4;
#pragma unroll
    for (int a = 0; a < 3; ++a) gg[1 + a][b] += -zm[a] + jm[a] * z4;
    gg[4][b] += j4 * z4;
    D0 += z4 * g[0][b];
#pragma unroll
    for (int a = 0; a < 3; ++a) Dm[a] += z4 * g[1 + a][b];
  }
  if (iso) {
    // d j0 / d rho = 2 U2 / rho, d j0 / d m_a = -2 U_a / rho; d jm_a / d rho = -2 U_a / rho,
    // d jm_a / d m_c = 2 delta_ac / rho
    R UDm = U[0] * Dm[0] + U[1] * Dm[1] + U[2] * Dm[2];
    gv[0] += R(2) * ir * (U2 * D0 - UDm);
#pragma unroll
    for (int a = 0; a < 3; ++a) gv[1 + a] += R(2) * ir * (Dm[a] - U[a] * D0);
  }
}

// Vector-Jacobian product of gp_flux_global: gacc[10] -> cotangents of vl, gl, vr, gr
// (accumulated).
template <class R>
GKS_HD bool gp_flux_global_vjp(const FluxParams<R>& P, const R vl[5], const R gl[5][3],
                               const R vr[5], const R gr[5][3], const R n1[3], R w, R dt,
                               const R gacc[10], R gvl[5], R ggl[5][3], R gvr[5], R ggr[5][3]) {
  int kk = 0;
  if (k_abs(n1[1]) < k_abs(n1[kk])) kk = 1;
  if (k_abs(n1[2]) < k_abs(n1[kk])) kk = 2;
  R n2[3];
  if (kk == 0) { n2[0] = R(0); n2[1] = n1[2]; n2[2] = -n1[1]; }
  else if (kk == 1) { n2[0] = -n1[2]; n2[1] = R(0); n2[2] = n1[0]; }
  else { n2[0] = n1[1]; n2[1] = -n1[0]; n2[2] = R(0); }
  const R il = R(1) / k_sqrt(n2[0] * n2[0] + n2[1] * n2[1] + n2[2] * n2[2]);
  n2[0] = n2[0] * il; n2[1] = n2[1] * il; n2[2] = n2[2] * il;
  const R n3[3] = {n1[1] * n2[2] - n1[2] * n2[1], n1[2] * n2[0] - n1[0] * n2[2],
                   n1[0] * n2[1] - n1[1] * n2[0]};
  const R* nm[3] = {n1, n2, n3};
  R ql[5], qr[5], dql[3][5], dqr[3][5];
  ql[0] = vl[0]; ql[4] = vl[4]; qr[0] = vr[0]; qr[4] = vr[4];
  for (int d = 0; d < 3; ++d) {
    ql[1 + d] = vl[1] * nm[d][0] + vl[2] * nm[d][1] + vl[3] * nm[d][2];
    qr[1 + d] = vr[1] * nm[d][0] + vr[2] * nm[d][1] + vr[3] * nm[d][2];
  }
  for (int d = 0; d < 3; ++d) {
    R sl[5], sr[5];
    for (int v = 0; v < 5; ++v) {
      sl[v] = gl[v][0] * nm[d][0] + gl[v][1] * nm[d][1] + gl[v][2] * nm[d][2];
      sr[v] = gr[v][0] * nm[d][0] + gr[v][1] * nm[d][1] + gr[v][2] * nm[d][2];
    }
    dql[d][0] = sl[0]; dql[d][4] = sl[4]; dqr[d][0] = sr[0]; dqr[d][4] = sr[4];
    for (int e = 0; e < 3; ++e) {
      dql[d][1 + e] = sl[1] * nm[e][0] + sl[2] * nm[e][1] + sl[3] * nm[e][2];
      dqr[d][1 + e] = sr[1] * nm[e][0] + sr[2] * nm[e][1] + sr[3] * nm[e][2];
    }
  }
  // back rotation and weight: acc = w [Fn0, sum_j Fn_j n_j, Fn4, Ft0, sum_j Ft_j n_j, Ft4]
  R gFn[5], gFt[5];
  gFn[0] = w * gacc[0];
  gFn[4] = w * gacc[4];
  gFt[0] = w * gacc[5];
  gFt[4] = w * gacc[9];
  for (int j = 0; j < 3; ++j) {
    gFn[1 + j] = w * (gacc[1] * nm[j][0] + gacc[2] * nm[j][1] + gacc[3] * nm[j][2]);
    gFt[1 + j] = w * (gacc[6] * nm[j][0] + gacc[7] * nm[j][1] + gacc[8] * nm[j][2]);
  }
  R gql[5] = {R(0), R(0), R(0), R(0), R(0)}, gqr[5] = {R(0), R(0), R(0), R(0), R(0)};
  R gdql[3][5], gdqr[3][5];
  for (int d = 0; d < 3; ++d)
    for (int v = 0; v < 5; ++v) gdql[d][v] = gdqr[d][v] = R(0);
  if (!gks_gp_flux_vjp_cf(P, ql, dql, qr, dqr, dt, gFn, gFt, gql, gdql, gqr, gdqr)) return false;
  // rotation into the local frame, reversed
  gvl[0] += gql[0]; gvl[4] += gql[4]; gvr[0] += gqr[0]; gvr[4] += gqr[4];
  for (int d = 0; d < 3; ++d)
    for (int a = 0; a < 3; ++a) {
      gvl[1 + a] += gql[1 + d] * nm[d][a];
      gvr[1 + a] += gqr[1 + d] * nm[d][a];
    }
  for (int d = 0; d < 3; ++d) {
    R gsl[5], gsr[5];
    gsl[0] = gdql[d][0]; gsl[4] = gdql[d][4]; gsr[0] = gdqr[d][0]; gsr[4] = gdqr[d][4];
    for (int b = 0; b < 3; ++b) {
      gsl[1 + b] = gdql[d][1] * nm[0][b] + gdql[d][2] * nm[1][b] + gdql[d][3] * nm[2][b];
      gsr[1 + b] = gdqr[d][1] * nm[0][b] + gdqr[d][2] * nm[1][b] + gdqr[d][3] * nm[2][b];
    }
    for (int v = 0; v < 5; ++v)
      for (int a = 0; a < 3; ++a) {
        ggl[v][a] += gsl[v] * nm[d][a];
        ggr[v][a] += gsr[v] * nm[d][a];
      }
  }
  return true;
}

// Adjoint of eval_poly: cotangents of value and gradient at offset d -> cotangents of the ten
// coefficients of each variable, gc[v][j] (accumulated).
template <class R>
GKS_HD void eval_poly_adj(const R d[3], const R gval[5], const R ggrad[5][3], R gc[5][10]) {
  const R xx = d[0] * d[0], yy = d[1] * d[1], zz = d[2] * d[2];
  const R xy = d[0] * d[1], xz = d[0] * d[2], yz = d[1] * d[2];
  for (int v = 0; v < 5; ++v) {
    const R g = gval[v], gx = ggrad[v][0], gy = ggrad[v][1], gz = ggrad[v][2];
    gc[v][0] += g;
    gc[v][1] += g * d[0] + gx;
    gc[v][2] += g * d[1] + gy;
    gc[v][3] += g * d[2] + gz;
    gc[v][4] += g * xx + R(2) * d[0] * gx;
    gc[v][5] += g * yy + R(2) * d[1] * gy;
    gc[v][6] += g * zz + R(2) * d[2] * gz;
    gc[v][7] += g * xy + d[1] * gx + d[0] * gy;
    gc[v][8] += g * xz + d[2] * gx + d[0] * gz;
    gc[v][9] += g * yz + d[2] * gy + d[1] * gz;
  }
}

}  // namespace gks

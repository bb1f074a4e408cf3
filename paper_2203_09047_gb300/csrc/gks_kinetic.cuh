// Gas-kinetic flux at one Gauss point (Section 3.2), written for the GPU: the half-space and
// interface-equilibrium moments in closed form, the slope terms as directional derivatives of
// closed-form moment vectors (no slope solve), and the time-fitted flux F^n, dF/dt.
#pragma once

#include <cuda_runtime.h>

#include <cmath>

#include "gks_internal.h"

namespace gks {

#define GKS_HD __host__ __device__ __forceinline__

GKS_HD double k_exp(double x) { return exp(x); }
GKS_HD float k_exp(float x) { return expf(x); }
GKS_HD double k_erfc(double x) { return erfc(x); }
GKS_HD float k_erfc(float x) { return erfcf(x); }
GKS_HD double k_sqrt(double x) { return sqrt(x); }
GKS_HD float k_sqrt(float x) { return sqrtf(x); }
GKS_HD double k_abs(double x) { return fabs(x); }
GKS_HD float k_abs(float x) { return fabsf(x); }
GKS_HD double k_pow(double x, double y) { return pow(x, y); }
GKS_HD float k_pow(float x, float y) { return powf(x, y); }
// Quotients of the per-state terms (reciprocals of rho and p, the half-line B, the frame
// normalisation, the pressure jump): the IEEE division, except for FP32 on the device, which
// takes the fast division intrinsic (within 2 ulp for divisors below 2^126). FP32 flux per
// launch, against IEEE divisions: smooth form 0.438 -> 0.421 ms on the 64^3-cube mesh, full
// form 6.52 -> 6.12 ms on the 128^3-cube explosion, 6.06 with the collision time and the
// time-fit quotients as well.
template <class R>
GKS_HD R k_div(R a, R b) {
  return a / b;
}
GKS_HD float k_div(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fdividef(a, b);
#else
  return a / b;
#endif
}

template <class R>
struct Prim {
  R rho, U, V, W, p, lam;
  R ir, ip, hil;  // 1/rho, 1/p, 1/(2 lam) = p/rho
};

// Primitives and the reciprocals the flux reuses (two divisions per state).
template <class R>
GKS_HD bool to_prim(const R q[5], R gamma, Prim<R>& w) {
  w.rho = q[0];
  w.ir = k_div(R(1), q[0]);
  w.U = q[1] * w.ir;
  w.V = q[2] * w.ir;
  w.W = q[3] * w.ir;
  w.p = (gamma - R(1)) * (q[4] - R(0.5) * (q[1] * w.U + q[2] * w.V + q[3] * w.W));
  w.ip = k_div(R(1), w.p);
  w.lam = R(0.5) * w.rho * w.ip;
  w.hil = w.p * w.ir;
  return (w.rho > R(0)) && (w.p > R(0));  // false also for NaN
}

// Moments of an equilibrium in closed form. For a Maxwellian g(W) of the conserved state W,
// dg = g (a . psi) with rho <a psi> = dW, so rho <c_d (a psi) psi> is the derivative of the
// Euler flux along axis d applied to dW. euler_flux_x: rho <u psi> = F_x(W).
// euler_jvp: A_d(W) dW = dF_d/dW dW, with dU = (dm - U drho)/rho and
// dp = (gamma - 1) (dE - U . dm + |U|^2 drho / 2).
template <class R>
GKS_HD void euler_flux_x(const Prim<R>& w, R E, R F[5]) {
  const R m = w.rho * w.U;
  F[0] = m;
  F[1] = m * w.U + w.p;
  F[2] = m * w.V;
  F[3] = m * w.W;
  F[4] = w.U * (E + w.p);
}
template <class R>
GKS_HD void euler_jvp(const Prim<R>& w, R ir, R gm1, R Ep, int d, const R dq[5], R out[5]) {
  const R U[3] = {w.U, w.V, w.W};
  const R du[3] = {(dq[1] - U[0] * dq[0]) * ir, (dq[2] - U[1] * dq[0]) * ir,
                   (dq[3] - U[2] * dq[0]) * ir};
  const R u2 = U[0] * U[0] + U[1] * U[1] + U[2] * U[2];
  const R dp = gm1 * (dq[4] - (U[0] * dq[1] + U[1] * dq[2] + U[2] * dq[3]) + R(0.5) * u2 * dq[0]);
  const R md = w.rho * U[d], dmd = dq[1 + d];
  out[0] = dmd;
#pragma unroll
  for (int a = 0; a < 3; ++a) out[1 + a] = dmd * U[a] + md * du[a];
  out[1 + d] += dp;
  out[4] = du[d] * Ep + U[d] * (dq[4] + dp);  // Ep = E + p
}

// Second-moment flux of an equilibrium along axis d, T_d(W) = rho <u c_d psi>, with theta = p/rho:
//   T_d[0]     = rho (U_0 U_d + theta delta_0d)
//   T_d[1 + a] = rho (U_0 U_d U_a + theta (U_0 delta_da + U_d delta_0a + U_a delta_0d))
//   T_d[4]     = rho/2 (U_0 U_d (|U|^2 + (K + 7) theta) + delta_0d theta (|U|^2 + (K + 5) theta))
// (u = c_0 the normal velocity). second_moment_jvp returns its derivative along the conserved
// increment dq, which equals rho <u c_d (a psi) psi> for the slope a with rho <a psi> = dq.
template <class R>
GKS_HD void second_moment_jvp(const Prim<R>& w, R ir, R gm1, R K, int d, const R dq[5], R out[5]) {
  const R U[3] = {w.U, w.V, w.W};
  const R dU[3] = {(dq[1] - U[0] * dq[0]) * ir, (dq[2] - U[1] * dq[0]) * ir,
                   (dq[3] - U[2] * dq[0]) * ir};
  const R q = U[0] * U[0] + U[1] * U[1] + U[2] * U[2];
  const R dp = gm1 * (dq[4] - (U[0] * dq[1] + U[1] * dq[2] + U[2] * dq[3]) + R(0.5) * q * dq[0]);
  const R th = w.p * ir;
  const R dth = (dp - th * dq[0]) * ir;
  const R dq2 = R(2) * (U[0] * dU[0] + U[1] * dU[1] + U[2] * dU[2]);
  const R Ud = U[d], dUd = dU[d];
  const R uu = U[0] * Ud, duu = dU[0] * Ud + U[0] * dUd;  // U_0 U_d and its derivative
  const R n = d == 0 ? R(1) : R(0);
  // per unit density: t and its derivative dt; out = drho t + rho dt
  R t[5], dt[5];
  t[0] = uu + th * n;
  dt[0] = duu + dth * n;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const R da = a == d ? R(1) : R(0), za = a == 0 ? R(1) : R(0);
    const R g = U[0] * da + Ud * za + U[a] * n, dg = dU[0] * da + dUd * za + dU[a] * n;
    t[1 + a] = uu * U[a] + th * g;
    dt[1 + a] = duu * U[a] + uu * dU[a] + dth * g + th * dg;
  }
  const R c7 = K + R(7), c5 = K + R(5);
  t[4] = R(0.5) * (uu * (q + c7 * th) + n * th * (q + c5 * th));
  dt[4] = R(0.5) * (duu * (q + c7 * th) + uu * (dq2 + c7 * dth) +
                    n * (dth * (q + c5 * th) + th * (dq2 + c5 * dth)));
#pragma unroll
  for (int k = 0; k < 5; ++k) out[k] = dq[0] * t[k] + w.rho * dt[k];
}

// Half-line equilibrium of one side (u > 0 for s = +1, u < 0 for s = -1; s is an int, or a
// packed pair of signs when R carries both sides) in closed form:
// A = <1>, A1 = <u>, A2 = <u^2> over the half line, B = exp(-lam U^2) / (2 sqrt(pi lam)) and
// S = <v^2 + w^2 + xi^2>, so that rho <psi> = rho (A, A1, V A, W A, (A2 + S A) / 2).
template <class R>
struct Half {
  R A, A1, A2, B, S;
};
template <class R, class Sg>
GKS_HD void half_init(const Prim<R>& w, R K, Sg s, Half<R>& h) {
  const R sl = k_sqrt(w.lam);
  h.A = R(0.5) * k_erfc(-R(s) * sl * w.U);
  h.B = k_div(R(0.28209479177387814) * k_exp(-w.lam * w.U * w.U), sl);  // 1/(2 sqrt(pi))
  h.A1 = w.U * h.A + R(s) * h.B;
  h.A2 = w.U * h.A1 + w.hil * h.A;
  h.S = w.V * w.V + w.W * w.W + (K + R(2)) * w.hil;
}
template <class R>
GKS_HD void half_moments(const Prim<R>& w, const Half<R>& h, R Q[5]) {
  Q[0] = w.rho * h.A;
  Q[1] = w.rho * h.A1;
  Q[2] = w.rho * w.V * h.A;
  Q[3] = w.rho * w.W * h.A;
  Q[4] = R(0.5) * w.rho * (h.A2 + h.S * h.A);
}
// Derivative of rho <psi> (half line) along the conserved increment dq, through the primitive
// increments dU = (dm - U drho)/rho, dp = (gamma - 1)(dE - U . dm + |U|^2 drho / 2),
// dlam/lam = drho/rho - dp/p, with dA = s B (2 lam dU + U dlam),
// dB = -B (2 lam U dU + (U^2 + 1/(2 lam)) dlam). Equals rho <a psi> (half line) for the slope a
// of the Maxwellian with rho <a psi> = dq over the full line. No division: the reciprocals come
// with the primitives.
template <class R, class Sg>
GKS_HD void half_jvp(const Prim<R>& w, R gm1, R K, Sg s, const Half<R>& h, const R dq[5],
                     R dQ[5]) {
  const R ir = w.ir, hil = w.hil;
  const R dU = (dq[1] - w.U * dq[0]) * ir, dV = (dq[2] - w.V * dq[0]) * ir,
          dW = (dq[3] - w.W * dq[0]) * ir;
  const R u2 = w.U * w.U + w.V * w.V + w.W * w.W;
  const R dp = gm1 * (dq[4] - (w.U * dq[1] + w.V * dq[2] + w.W * dq[3]) + R(0.5) * u2 * dq[0]);
  const R dll = dq[0] * ir - dp * w.ip;  // dlam / lam
  const R dlam = w.lam * dll;
  const R dA = R(s) * h.B * (R(2) * w.lam * dU + w.U * dlam);
  const R dB = -h.B * (R(2) * w.lam * w.U * dU + (w.U * w.U + hil) * dlam);
  const R dA1 = dU * h.A + w.U * dA + R(s) * dB;
  const R dA2 = dU * h.A1 + w.U * dA1 + hil * (dA - h.A * dll);
  const R dS = R(2) * (w.V * dV + w.W * dW) - (K + R(2)) * hil * dll;
  dQ[0] = dq[0] * h.A + w.rho * dA;
  dQ[1] = dq[0] * h.A1 + w.rho * dA1;
  dQ[2] = dq[0] * w.V * h.A + w.rho * (dV * h.A + w.V * dA);
  dQ[3] = dq[0] * w.W * h.A + w.rho * (dW * h.A + w.W * dA);
  dQ[4] = R(0.5) * (dq[0] * (h.A2 + h.S * h.A) + w.rho * (dA2 + dS * h.A + h.S * dA));
}

// Half-line flux terms of the full flux in closed form. With the half-line moments
// A_n = <u^n> (n = 0..4, A_{n+2} = U A_{n+1} + (n + 1) A_n / (2 lam)), the full-line moments of
// v, w and xi^2 = K / (2 lam):
//   F+(W)    = rho <u psi>     = rho (A1, A2, V A1, W A1, (A3 + S A1) / 2),
//   T+_0(W)  = rho <u u psi>   = rho (A2, A3, V A2, W A2, (A4 + S A2) / 2),
//   T+_1(W)  = rho <u v psi>   = rho (V A1, V A2, <v^2> A1, V W A1, (V A3 + Y_v A1) / 2),
//   T+_2(W)  = rho <u w psi>   = rho (W A1, W A2, V W A1, <w^2> A1, (W A3 + Y_w A1) / 2),
// S = V^2 + W^2 + (K + 2)/(2 lam), Y_v = V (V^2 + W^2 + (K + 4)/(2 lam)), Y_w likewise. Their
// derivatives along a conserved increment dW are the half-line slope terms of Eq. flux-1:
// rho <u (a psi) psi>_+ = DF+[dW] and rho <u c_d (a psi) psi>_+ = DT+_d[dW] for the slope a with
// rho <a psi> = dW.
template <class R>
struct HalfLine {
  R A[5], B;
};
template <class R>
GKS_HD void half_line(const Prim<R>& w, const Half<R>& h, HalfLine<R>& m) {
  m.A[0] = h.A;
  m.A[1] = h.A1;
  m.A[2] = h.A2;
  m.A[3] = w.U * m.A[2] + R(2) * w.hil * m.A[1];
  m.A[4] = w.U * m.A[3] + R(3) * w.hil * m.A[2];
  m.B = h.B;
}
// Primitive increments along dq and the half-line moment increments dA[0..4].
template <class R>
struct DPrim {
  R drho, dU, dV, dW, dlam, dhil;
};
template <class R>
GKS_HD void dprim(const Prim<R>& w, R gm1, const R dq[5], DPrim<R>& d) {
  const R ir = w.ir;
  d.drho = dq[0];
  d.dU = (dq[1] - w.U * dq[0]) * ir;
  d.dV = (dq[2] - w.V * dq[0]) * ir;
  d.dW = (dq[3] - w.W * dq[0]) * ir;
  const R u2 = w.U * w.U + w.V * w.V + w.W * w.W;
  const R dp = gm1 * (dq[4] - (w.U * dq[1] + w.V * dq[2] + w.W * dq[3]) + R(0.5) * u2 * dq[0]);
  const R dll = dq[0] * ir - dp * w.ip;  // dlam / lam
  d.dlam = w.lam * dll;
  d.dhil = -w.hil * dll;
}
template <class R, class Sg>
GKS_HD void dhalf_line(const Prim<R>& w, Sg s, const HalfLine<R>& m, const DPrim<R>& d,
                       R dA[5]) {
  const R U = w.U, hil = w.hil;
  dA[0] = R(s) * m.B * (R(2) * w.lam * d.dU + U * d.dlam);
  const R dB = -m.B * (R(2) * w.lam * U * d.dU + (U * U + hil) * d.dlam);
  dA[1] = d.dU * m.A[0] + U * dA[0] + R(s) * dB;
  dA[2] = d.dU * m.A[1] + U * dA[1] + d.dhil * m.A[0] + hil * dA[0];
  dA[3] = d.dU * m.A[2] + U * dA[2] + R(2) * (d.dhil * m.A[1] + hil * dA[1]);
  dA[4] = d.dU * m.A[3] + U * dA[3] + R(3) * (d.dhil * m.A[2] + hil * dA[2]);
}
template <class R>
GKS_HD void half_flux(const Prim<R>& w, R K, const HalfLine<R>& m, R F[5]) {
  const R S = w.V * w.V + w.W * w.W + (K + R(2)) * w.hil;
  F[0] = w.rho * m.A[1];
  F[1] = w.rho * m.A[2];
  F[2] = w.rho * w.V * m.A[1];
  F[3] = w.rho * w.W * m.A[1];
  F[4] = R(0.5) * w.rho * (m.A[3] + S * m.A[1]);
}
// DF+[dq]
template <class R, class Sg>
GKS_HD void half_flux_jvp(const Prim<R>& w, R gm1, R K, Sg s, const HalfLine<R>& m,
                          const R dq[5], R out[5]) {
  DPrim<R> d;
  dprim(w, gm1, dq, d);
  R dA[5];
  dhalf_line(w, s, m, d, dA);
  const R S = w.V * w.V + w.W * w.W + (K + R(2)) * w.hil;
  const R dS = R(2) * (w.V * d.dV + w.W * d.dW) + (K + R(2)) * d.dhil;
  out[0] = d.drho * m.A[1] + w.rho * dA[1];
  out[1] = d.drho * m.A[2] + w.rho * dA[2];
  out[2] = d.drho * w.V * m.A[1] + w.rho * (d.dV * m.A[1] + w.V * dA[1]);
  out[3] = d.drho * w.W * m.A[1] + w.rho * (d.dW * m.A[1] + w.W * dA[1]);
  out[4] = R(0.5) * (d.drho * (m.A[3] + S * m.A[1]) +
                     w.rho * (dA[3] + dS * m.A[1] + S * dA[1]));
}
// DT+_k[dq] for the velocity component k (0 normal, 1, 2 tangential)
template <class R, class Sg>
GKS_HD void half_second_jvp(const Prim<R>& w, R gm1, R K, Sg s, const HalfLine<R>& m, int k,
                            const R dq[5], R out[5]) {
  DPrim<R> d;
  dprim(w, gm1, dq, d);
  R dA[5];
  dhalf_line(w, s, m, d, dA);
  const R V = w.V, W = w.W, hil = w.hil;
  R t[5], dt[5];
  if (k == 0) {
    const R S = V * V + W * W + (K + R(2)) * hil;
    const R dS = R(2) * (V * d.dV + W * d.dW) + (K + R(2)) * d.dhil;
    t[0] = m.A[2];
    dt[0] = dA[2];
    t[1] = m.A[3];
    dt[1] = dA[3];
    t[2] = V * m.A[2];
    dt[2] = d.dV * m.A[2] + V * dA[2];
    t[3] = W * m.A[2];
    dt[3] = d.dW * m.A[2] + W * dA[2];
    t[4] = R(0.5) * (m.A[4] + S * m.A[2]);
    dt[4] = R(0.5) * (dA[4] + dS * m.A[2] + S * dA[2]);
  } else {
    // c = the tangential component k, o = the other one
    const R c = k == 1 ? V : W, o = k == 1 ? W : V;
    const R dc = k == 1 ? d.dV : d.dW, dO = k == 1 ? d.dW : d.dV;
    const R c2 = c * c + hil, dc2 = R(2) * c * dc + d.dhil;  // <c^2>
    const R q = V * V + W * W + (K + R(4)) * hil;
    const R dqq = R(2) * (V * d.dV + W * d.dW) + (K + R(4)) * d.dhil;
    const R Y = c * q, dY = dc * q + c * dqq;
    t[0] = c * m.A[1];
    dt[0] = dc * m.A[1] + c * dA[1];
    t[1] = c * m.A[2];
    dt[1] = dc * m.A[2] + c * dA[2];
    // momentum components along this tangential axis and the other one
    const R tc = c2 * m.A[1], dtc = dc2 * m.A[1] + c2 * dA[1];
    const R to = c * o * m.A[1], dto = (dc * o + c * dO) * m.A[1] + c * o * dA[1];
    t[2] = k == 1 ? tc : to;
    dt[2] = k == 1 ? dtc : dto;
    t[3] = k == 1 ? to : tc;
    dt[3] = k == 1 ? dto : dtc;
    t[4] = R(0.5) * (c * m.A[3] + Y * m.A[1]);
    dt[4] = R(0.5) * (dc * m.A[3] + c * dA[3] + dY * m.A[1] + Y * dA[1]);
  }
#pragma unroll
  for (int q2 = 0; q2 < 5; ++q2) out[q2] = d.drho * t[q2] + w.rho * dt[q2];
}

template <class R>
struct FluxParams {
  R gamma, K, mu, tau_eps, tau_C;
  int full, tau_model;
  R pr_fix = R(0);  // 1/Pr - 1 (heat-flux correction of the smooth flux; 0 for the BGK value)
  R T_ref = R(1), mu_pow = R(0.7);  // power law mu (T / T_ref)^mu_pow (collision time 3)
};

// One boundary plane: no-slip wall velocity and temperature (<= 0: adiabatic), far-field state
// (rho, U, V, W, p). The kernels read it from a [6][kPlaneStride] device table (plane axis +
// 3 side: uw[3], Tw, finf[5], padding) only at boundary faces, so that the parameter block
// holds no array indexed at run time.
template <class R>
struct WallData {
  R uw[3] = {R(0), R(0), R(0)};
  R Tw = R(0);
  const R* finf = nullptr;  // far-field planes: (rho, U, V, W, p) in the table
};
template <class R>
GKS_HD WallData<R> wall_data(const R* table, int code) {
  WallData<R> d;
  if (code >= 6) {
    const R* t = table + kPlaneStride * (code % 6);
#pragma unroll
    for (int a = 0; a < 3; ++a) d.uw[a] = t[a];
    d.Tw = t[3];
    d.finf = t + 4;
  }
  return d;
}

// Flux parameters from the solver's kernel parameters (any struct with the same field names).
template <class R, template <class> class KP>
inline FluxParams<R> flux_params(const KP<R>& p) {
  FluxParams<R> fp;
  fp.gamma = p.gamma;
  fp.K = p.K;
  fp.mu = p.mu;
  fp.tau_eps = p.tau_eps;
  fp.tau_C = p.tau_C;
  fp.full = p.flux_mode;
  fp.tau_model = p.tau_model;
  fp.pr_fix = p.pr_fix;
  fp.T_ref = p.T_ref;
  fp.mu_pow = p.mu_pow;
  return fp;
}

// Collision time of the interface (Section 5): zero; inviscid (eps + C dp) dt; viscous
// mu / p0 + C dp dt, with mu constant or the power law of Section 5.4 at T0 = p0 / rho0.
template <class R>
GKS_HD R collision_time(const FluxParams<R>& P, R p0, R ir0, R dp, R dt) {
  if (P.tau_model == 1) return (P.tau_eps + P.tau_C * dp) * dt;
  if (P.tau_model == 2) return k_div(P.mu, p0) + P.tau_C * dp * dt;
  if (P.tau_model == 3)
    return k_div(P.mu * k_pow(k_div(p0 * ir0, P.T_ref), P.mu_pow), p0) + P.tau_C * dp * dt;
  return R(0);
}

// Far-field state at a plane of axis ax with outward normal sign sg (Section 5.4, Riemann
// invariants): R+ = u_n + 2c/(gamma-1) from the inside state q, R- = u_n - 2c/(gamma-1) from
// the far field; u_n and c of the boundary are their mean and (gamma-1)/4 of their difference;
// entropy p/rho^gamma and tangential velocity from the upwind side; supersonic inflow takes the
// far field, supersonic outflow q. Conserved variables in and out.
template <class R>
GKS_HD void farfield_state(const FluxParams<R>& P, const R finf[5], int ax, R sg, const R q[5],
                           R out[5]) {
  const R g = P.gamma, gm1 = P.gamma - R(1);
  const R ir = R(1) / q[0];
  const R U[3] = {q[1] * ir, q[2] * ir, q[3] * ir};
  const R p = gm1 * (q[4] - R(0.5) * (q[1] * U[0] + q[2] * U[1] + q[3] * U[2]));
  const R c = k_sqrt(g * p * ir);
  const R un = sg * U[ax];
  const R rinf = finf[0], pinf = finf[4];
  const R Uinf[3] = {finf[1], finf[2], finf[3]};
  const R uninf = sg * Uinf[ax];
  const R cinf = k_sqrt(g * pinf / rinf);
  R rb, pb, Ub[3];
  if (un >= c) {
#pragma unroll
    for (int v = 0; v < 5; ++v) out[v] = q[v];
    return;
  }
  if (un <= -c) {
    rb = rinf;
    pb = pinf;
#pragma unroll
    for (int a = 0; a < 3; ++a) Ub[a] = Uinf[a];
  } else {
    const R Rp = un + R(2) * c / gm1, Rm = uninf - R(2) * cinf / gm1;
    const R unb = R(0.5) * (Rp + Rm), cb = R(0.25) * gm1 * (Rp - Rm);
    const bool out_flow = unb >= R(0);
    const R s = out_flow ? p / k_pow(q[0], g) : pinf / k_pow(rinf, g);
#pragma unroll
    for (int a = 0; a < 3; ++a) Ub[a] = out_flow ? U[a] : Uinf[a];
    Ub[ax] = sg * unb;  // tangential components kept, the normal one from the invariants
    rb = k_pow(cb * cb / (g * s), R(1) / gm1);
    pb = rb * cb * cb / g;
  }
  out[0] = rb;
#pragma unroll
  for (int a = 0; a < 3; ++a) out[1 + a] = rb * Ub[a];
  out[4] = pb / gm1 + R(0.5) * rb * (Ub[0] * Ub[0] + Ub[1] * Ub[1] + Ub[2] * Ub[2]);
}

// Ghost value and gradient at a Gauss point of wall `code` (global frame; code as in
// gks_internal.h: axis + 3 side, + 6 for a no-slip wall). Geometry is mirrored (d/dx_axis
// changes sign); the flow variables: slip, the normal momentum negated; no-slip with (U_w, T_w),
// rho_g = rho, m_g = 2 U_w rho - m and E_g = E + 2 |U_w|^2 rho - 2 U_w . m (adiabatic, p_g = p)
// or E_g = 2 rho T_w / (gamma-1) - E + |m|^2/rho + 2 |U_w|^2 rho - 2 U_w . m (isothermal,
// T_g = 2 T_w - T); the gradient is mapped by the Jacobian of that map.
// kFar = false leaves the far-field branch out (for callers that never see far-field planes).
template <class R, bool kFar = true>
GKS_HD void wall_ghost(const FluxParams<R>& P, int code, const WallData<R>& wd, const R v[5],
                       const R g[5][3], R vg[5], R gg[5][3]) {
  const int ax = code % 3;
  if (kFar && code >= 12) {  // far field: the characteristic state, uniform
    farfield_state(P, wd.finf, ax, (code % 6) >= 3 ? R(1) : R(-1), v, vg);
#pragma unroll
    for (int r = 0; r < 5; ++r)
#pragma unroll
      for (int b = 0; b < 3; ++b) gg[r][b] = R(0);
    return;
  }
  if (code < 6) {
#pragma unroll
    for (int r = 0; r < 5; ++r) {
      const R sv = (r == 1 + ax) ? R(-1) : R(1);
      vg[r] = sv * v[r];
#pragma unroll
      for (int b = 0; b < 3; ++b) gg[r][b] = (b == ax ? -sv : sv) * g[r][b];
    }
    return;
  }
  const R u0 = wd.uw[0], u1 = wd.uw[1], u2 = wd.uw[2], Tw = wd.Tw;
  const R uw2 = u0 * u0 + u1 * u1 + u2 * u2;
  const R uw[3] = {u0, u1, u2};
  // row 4 of the Jacobian: dE_g = j0 drho + jm . dm + j4 dE
  R j0, jm[3], j4;
  const R rho = v[0];
  const R um = u0 * v[1] + u1 * v[2] + u2 * v[3];
  if (Tw > R(0)) {
    const R ir = R(1) / rho;
    const R U[3] = {v[1] * ir, v[2] * ir, v[3] * ir};
    const R U2 = U[0] * U[0] + U[1] * U[1] + U[2] * U[2];
    const R cT = R(2) * Tw / (P.gamma - R(1));
    vg[4] = cT * rho - v[4] + U2 * rho + R(2) * uw2 * rho - R(2) * um;
    j0 = cT - U2 + R(2) * uw2;
#pragma unroll
    for (int a = 0; a < 3; ++a) jm[a] = R(2) * (U[a] - uw[a]);
    j4 = R(-1);
  } else {
    vg[4] = v[4] + R(2) * uw2 * rho - R(2) * um;
    j0 = R(2) * uw2;
#pragma unroll
    for (int a = 0; a < 3; ++a) jm[a] = R(-2) * uw[a];
    j4 = R(1);
  }
  vg[0] = rho;
#pragma unroll
  for (int a = 0; a < 3; ++a) vg[1 + a] = R(2) * uw[a] * rho - v[1 + a];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const R sb = b == ax ? R(-1) : R(1);
    gg[0][b] = sb * g[0][b];
#pragma unroll
    for (int a = 0; a < 3; ++a) gg[1 + a][b] = sb * (R(2) * uw[a] * g[0][b] - g[1 + a][b]);
    gg[4][b] = sb * (j0 * g[0][b] + jm[0] * g[1][b] + jm[1] * g[2][b] + jm[2] * g[3][b] +
                     j4 * g[4][b]);
  }
}

// The wall flux (after the Gauss-point sum): no mass; a slip wall passes normal momentum only;
// an adiabatic no-slip wall conducts no heat, so its energy flux is U_w . (momentum flux).
template <class R>
GKS_HD void wall_flux_fix(int code, const WallData<R>& wd, R acc[10]) {
  if (code >= 12) return;  // a far-field plane passes the GKS flux of its ghost pair
  acc[0] = acc[5] = R(0);
  const int ax = code % 3;
  if (code < 6) {
#pragma unroll
    for (int v = 1; v < 5; ++v)
      if (v != 1 + ax) acc[v] = acc[5 + v] = R(0);
    return;
  }
  if (wd.Tw <= R(0)) {
    acc[4] = wd.uw[0] * acc[1] + wd.uw[1] * acc[2] + wd.uw[2] * acc[3];
    acc[9] = wd.uw[0] * acc[6] + wd.uw[1] * acc[7] + wd.uw[2] * acc[8];
  }
}

// Time integrals over [0, d] of the six coefficients of Eq. flux-1.
template <class R>
GKS_HD void flux1_integrals(R tau, R d, R c[6]) {
  const R e = k_exp(k_div(-d, tau));
  const R om = R(1) - e;
  c[0] = d - tau * om;
  c[1] = R(2) * tau * tau * om - tau * d * (R(1) + e);
  c[2] = R(0.5) * d * d - tau * d + tau * tau * om;
  c[3] = tau * om;
  c[4] = tau * d * e - R(2) * tau * tau * om;
  c[5] = -tau * tau * om;
}

// Interface-equilibrium terms of both flux forms from the interface state Q0 (primitives w0)
// and its conserved-variable slopes dW_d along the local axes: the equilibrium time slope
// rho0 <Ab psi>_0 = -sum_d rho0 <c_d ab_d psi>_0 = -sum_d A_d dW_d, the flux moments
// E0 = rho0 <u psi>_0, E1 = rho0 <u (ab . c) psi>_0 = sum_d D T_d(W0)[dW_d] (only with a
// collision-time model; zero otherwise, where tau = 0 multiplies it) and
// E2 = rho0 <u Ab psi>_0 = A_x dWt, and the collision time from the two sides' pressures.
template <class R>
GKS_HD void interface_terms(const FluxParams<R>& P, R pl, R pr, const R q0[5], const Prim<R>& w0,
                            const R dW[3][5], R dt, R dWt[5], R E0[5], R E1[5], R E2[5],
                            R& tau) {
  const R gm1 = P.gamma - R(1);
  const R ir0 = w0.ir, Ep0 = q0[4] + w0.p;
  R t[5];
  euler_jvp(w0, ir0, gm1, Ep0, 0, dW[0], dWt);
  euler_jvp(w0, ir0, gm1, Ep0, 1, dW[1], t);
#pragma unroll
  for (int q = 0; q < 5; ++q) dWt[q] += t[q];
  euler_jvp(w0, ir0, gm1, Ep0, 2, dW[2], t);
#pragma unroll
  for (int q = 0; q < 5; ++q) dWt[q] = -(dWt[q] + t[q]);
  euler_flux_x(w0, q0[4], E0);
  euler_jvp(w0, ir0, gm1, Ep0, 0, dWt, E2);
  const R dp = k_abs(k_div(pl - pr, pl + pr));
  tau = collision_time(P, w0.p, ir0, dp, dt);
  if (P.tau_model != 0) {
    second_moment_jvp(w0, ir0, gm1, P.K, 0, dW[0], E1);
#pragma unroll
    for (int d = 1; d < 3; ++d) {
      second_moment_jvp(w0, ir0, gm1, P.K, d, dW[d], t);
#pragma unroll
      for (int q = 0; q < 5; ++q) E1[q] += t[q];
    }
  } else {
#pragma unroll
    for (int q = 0; q < 5; ++q) E1[q] = R(0);
  }
}

// Smooth flux (Eq. flux-2) from the interface terms: F(delta) = E0 delta - tau delta (E1 + E2)
// + delta^2/2 E2, so the two-point time fit is exact; with the heat-flux correction the energy
// components gain pr_fix times the heat flux relative to the interface velocity, from the flux
// moments F and the conserved moments m of the time-integrated distribution (m^n = Q0,
// dm/dt = dWt; the tau terms of m vanish by the compatibility condition defining Ab).
template <class R>
GKS_HD void smooth_from_terms(const FluxParams<R>& P, const R q0[5], const Prim<R>& w0,
                              const R dWt[5], const R E0[5], const R E1[5], const R E2[5], R tau,
                              R Fn[5], R Ft[5]) {
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    Fn[q] = E0[q] - tau * (E1[q] + E2[q]);
    Ft[q] = E2[q];
  }
  if (P.pr_fix != R(0)) {
    const R u2 = w0.U * w0.U + w0.V * w0.V + w0.W * w0.W;
    auto heat = [&](const R F[5], const R m[5]) {
      return F[4] - (w0.U * F[1] + w0.V * F[2] + w0.W * F[3]) + R(0.5) * u2 * F[0] -
             (w0.U * m[4] - w0.U * (w0.U * m[1] + w0.V * m[2] + w0.W * m[3]) +
              R(0.5) * w0.U * u2 * m[0]);
    };
    const R qn = heat(Fn, q0);
    const R qt = heat(Ft, dWt);
    Fn[4] += P.pr_fix * qn;
    Ft[4] += P.pr_fix * qt;
  }
}

// Coefficients of the two-point time fit of the full flux: F^n and dF/dt are sums over the six
// terms of Eq. flux-1 with weights cn and ct from the time integrals over [0, dt/2] and [0, dt]
// (tau = 0: the equilibrium flux and its time derivative alone).
template <class R>
GKS_HD void full_fit_coeffs(R tau, R dt, R cn[6], R ct[6]) {
  if (tau > R(0)) {
    R ch[6], cf[6];
    flux1_integrals(tau, R(0.5) * dt, ch);
    flux1_integrals(tau, dt, cf);
    const R idt = k_div(R(1), dt);
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      cn[q] = (R(4) * ch[q] - cf[q]) * idt;
      ct[q] = R(4) * (cf[q] - R(2) * ch[q]) * idt * idt;
    }
  } else {
#pragma unroll
    for (int q = 0; q < 6; ++q) cn[q] = ct[q] = R(0);
    cn[0] = R(1);
    ct[2] = R(1);
  }
}

// Gauss-point flux in the local frame (u along the normal). ql/qr: conserved states;
// dql/dqr[m]: their derivatives along n1, n2, n3 (momentum already in the local frame).
// Writes Fn = F^n and Ft = dF/dt of the two-point time fit. Returns false for a non-physical
// state.
template <class R>
GKS_HD bool gks_gp_flux(const FluxParams<R>& P, const R ql[5],
                                            const R dql[3][5], const R qr[5], const R dqr[3][5],
                                            R dt, R Fn[5], R Ft[5]) {
  Prim<R> wl, wr, w0;
  bool ok = to_prim(ql, P.gamma, wl) & to_prim(qr, P.gamma, wr);
  if (!ok) return false;
  const R gm1 = P.gamma - R(1);
  Half<R> hl, hr;
  half_init(wl, P.K, +1, hl);
  half_init(wr, P.K, -1, hr);
  // interface equilibrium Q0 from the two half-space moments
  R q0[5], t[5];
  half_moments(wl, hl, q0);
  half_moments(wr, hr, t);
#pragma unroll
  for (int q = 0; q < 5; ++q) q0[q] += t[q];
  if (!to_prim(q0, P.gamma, w0)) return false;
  // conserved-variable slopes of the interface equilibrium, dW_d = rho0 <ab_d psi>_0: the
  // half-space parts rho <a_d psi>_{u>0} + rho <a_d psi>_{u<0} of both sides' slopes
  const R irl = wl.ir, irr = wr.ir;
  R dW[3][5];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    half_jvp(wl, gm1, P.K, +1, hl, dql[d], dW[d]);
    half_jvp(wr, gm1, P.K, -1, hr, dqr[d], t);
#pragma unroll
    for (int q = 0; q < 5; ++q) dW[d][q] += t[q];
  }
  R dWt[5], E0[5], E1[5], E2[5], tau;
  interface_terms(P, wl.p, wr.p, q0, w0, dW, dt, dWt, E0, E1, E2, tau);
  if (!P.full) {
    smooth_from_terms(P, q0, w0, dWt, E0, E1, E2, tau, Fn, Ft);
    return true;
  }
  // full flux: the non-equilibrium parts of both sides. With the side's slopes a_d (rho <a_d psi>
  // = dq_d) and time slope A (rho <A psi> = -sum_d A_d(W) dq_d, Euler Jacobians at the side's
  // state): N0 = F+(W), N1 = sum_d DT+_d[dq_d] = rho <u (a . c) psi>_+, N2 = DF+[rho <A psi>]
  // = rho <u A psi>_+ (half line u > 0 on the left, u < 0 on the right)
  R NL[3][5], NR[3][5];
  {
    HalfLine<R> ml, mr;
    half_line(wl, hl, ml);
    half_line(wr, hr, mr);
    half_flux(wl, P.K, ml, NL[0]);
    half_flux(wr, P.K, mr, NR[0]);
    R dtl[5], dtr[5];
    const R Epl = ql[4] + wl.p, Epr = qr[4] + wr.p;
    euler_jvp(wl, irl, gm1, Epl, 0, dql[0], dtl);
    euler_jvp(wr, irr, gm1, Epr, 0, dqr[0], dtr);
    half_second_jvp(wl, gm1, P.K, +1, ml, 0, dql[0], NL[1]);
    half_second_jvp(wr, gm1, P.K, -1, mr, 0, dqr[0], NR[1]);
#pragma unroll
    for (int d = 1; d < 3; ++d) {
      euler_jvp(wl, irl, gm1, Epl, d, dql[d], t);
#pragma unroll
      for (int q = 0; q < 5; ++q) dtl[q] += t[q];
      euler_jvp(wr, irr, gm1, Epr, d, dqr[d], t);
#pragma unroll
      for (int q = 0; q < 5; ++q) dtr[q] += t[q];
      half_second_jvp(wl, gm1, P.K, +1, ml, d, dql[d], t);
#pragma unroll
      for (int q = 0; q < 5; ++q) NL[1][q] += t[q];
      half_second_jvp(wr, gm1, P.K, -1, mr, d, dqr[d], t);
#pragma unroll
      for (int q = 0; q < 5; ++q) NR[1][q] += t[q];
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      dtl[q] = -dtl[q];
      dtr[q] = -dtr[q];
    }
    half_flux_jvp(wl, gm1, P.K, +1, ml, dtl, NL[2]);
    half_flux_jvp(wr, gm1, P.K, -1, mr, dtr, NR[2]);
  }
  R cn[6], ct[6];
  full_fit_coeffs(tau, dt, cn, ct);
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const R geq_n = cn[0] * E0[q] + cn[1] * E1[q] + cn[2] * E2[q];
    const R geq_t = ct[0] * E0[q] + ct[1] * E1[q] + ct[2] * E2[q];
    const R gl_n = cn[3] * NL[0][q] + cn[4] * NL[1][q] + cn[5] * NL[2][q];
    const R gl_t = ct[3] * NL[0][q] + ct[4] * NL[1][q] + ct[5] * NL[2][q];
    const R gr_n = cn[3] * NR[0][q] + cn[4] * NR[1][q] + cn[5] * NR[2][q];
    const R gr_t = ct[3] * NR[0][q] + ct[4] * NR[1][q] + ct[5] * NR[2][q];
    Fn[q] = geq_n + gl_n + gr_n;
    Ft[q] = geq_t + gl_t + gr_t;
  }
  return true;
}

// The ten coefficients of variable v through the accessor; accessors over device memory
// provide their own (vector-load) version, found by argument-dependent lookup.
template <class Coef, class R>
GKS_HD void load_coefs(const Coef& coef, int v, R k[10]) {
#pragma unroll
  for (int j = 0; j < 10; ++j) k[j] = coef(v, j);
}

// Value and gradient at offset d of a cell polynomial c[v][j] in physical offsets from the
// centroid: Q = c0 + c1 dx + c2 dy + c3 dz + c4 dx^2 + c5 dy^2 + c6 dz^2 + c7 dxdy + c8 dxdz
// + c9 dydz. `coef(v, j)` returns coefficient j of variable v.
template <class R, class Coef>
GKS_HD void eval_poly(const Coef& coef, const R d[3], R val[5], R grad[5][3]) {
  const R xx = d[0] * d[0], yy = d[1] * d[1], zz = d[2] * d[2];
  const R xy = d[0] * d[1], xz = d[0] * d[2], yz = d[1] * d[2];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    R k[10];
    load_coefs(coef, v, k);
    val[v] = k[0] + k[1] * d[0] + k[2] * d[1] + k[3] * d[2] + k[4] * xx + k[5] * yy + k[6] * zz +
             k[7] * xy + k[8] * xz + k[9] * yz;
    grad[v][0] = k[1] + R(2) * k[4] * d[0] + k[7] * d[1] + k[8] * d[2];
    grad[v][1] = k[2] + R(2) * k[5] * d[1] + k[7] * d[0] + k[9] * d[2];
    grad[v][2] = k[3] + R(2) * k[6] * d[2] + k[8] * d[0] + k[9] * d[1];
  }
}

// The local frame of a Gauss point: n1 the unit normal, n2 = n1 x e_k / |n1 x e_k| with e_k the
// axis least aligned with n1, n3 = n1 x n2.
template <class R>
GKS_HD void face_frame(const R n1[3], R n2[3], R n3[3]) {
  int kk = 0;
  if (k_abs(n1[1]) < k_abs(n1[kk])) kk = 1;
  if (k_abs(n1[2]) < k_abs(n1[kk])) kk = 2;
  if (kk == 0) { n2[0] = R(0); n2[1] = n1[2]; n2[2] = -n1[1]; }
  else if (kk == 1) { n2[0] = -n1[2]; n2[1] = R(0); n2[2] = n1[0]; }
  else { n2[0] = n1[1]; n2[1] = -n1[0]; n2[2] = R(0); }
  const R il = k_div(R(1), k_sqrt(n2[0] * n2[0] + n2[1] * n2[1] + n2[2] * n2[2]));
  n2[0] = n2[0] * il; n2[1] = n2[1] * il; n2[2] = n2[2] * il;
  n3[0] = n1[1] * n2[2] - n1[2] * n2[1];
  n3[1] = n1[2] * n2[0] - n1[0] * n2[2];
  n3[2] = n1[0] * n2[1] - n1[1] * n2[0];
}

// A local-frame flux (F^n, dF/dt) rotated back to the global frame and weighted by the
// quadrature weight w: acc[0..4] = w F^n, acc[5..9] = w dF/dt.
template <class R>
GKS_HD void rotate_flux_out(const R Fn[5], const R Ft[5], const R n1[3], const R n2[3],
                            const R n3[3], R w, R acc[10]) {
  acc[0] = w * Fn[0];
  acc[4] = w * Fn[4];
  acc[5] = w * Ft[0];
  acc[9] = w * Ft[4];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    acc[1 + a] = w * (Fn[1] * n1[a] + Fn[2] * n2[a] + Fn[3] * n3[a]);
    acc[6 + a] = w * (Ft[1] * n1[a] + Ft[2] * n2[a] + Ft[3] * n3[a]);
  }
}

// Whole Gauss-point contribution in the global frame. Left/right values and gradients are
// rotated into the local frame (n1 the unit normal, n2 = n1 x e_k / |n1 x e_k| with e_k the axis
// least aligned with n1, n3 = n1 x n2), the local flux is computed, rotated back and multiplied
// by the quadrature weight w: acc[0..4] = w F^n, acc[5..9] = w dF/dt.
template <class R>
GKS_HD bool gp_flux_global(const FluxParams<R>& P, const R vl[5], const R gl[5][3], const R vr[5],
                           const R gr[5][3], const R n1[3], R w, R dt, R acc[10]) {
  R n2[3], n3[3];
  face_frame(n1, n2, n3);
  const R* nm[3] = {n1, n2, n3};
  R ql[5], qr[5], dql[3][5], dqr[3][5];
  ql[0] = vl[0]; ql[4] = vl[4]; qr[0] = vr[0]; qr[4] = vr[4];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    ql[1 + d] = vl[1] * nm[d][0] + vl[2] * nm[d][1] + vl[3] * nm[d][2];
    qr[1 + d] = vr[1] * nm[d][0] + vr[2] * nm[d][1] + vr[3] * nm[d][2];
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    R sl[5], sr[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      sl[v] = gl[v][0] * nm[d][0] + gl[v][1] * nm[d][1] + gl[v][2] * nm[d][2];
      sr[v] = gr[v][0] * nm[d][0] + gr[v][1] * nm[d][1] + gr[v][2] * nm[d][2];
    }
    dql[d][0] = sl[0]; dql[d][4] = sl[4]; dqr[d][0] = sr[0]; dqr[d][4] = sr[4];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      dql[d][1 + e] = sl[1] * nm[e][0] + sl[2] * nm[e][1] + sl[3] * nm[e][2];
      dqr[d][1 + e] = sr[1] * nm[e][0] + sr[2] * nm[e][1] + sr[3] * nm[e][2];
    }
  }
  R Fn[5], Ft[5];
  if (!gks_gp_flux(P, ql, dql, qr, dqr, dt, Fn, Ft)) return false;
  rotate_flux_out(Fn, Ft, n1, n2, n3, w, acc);
  return true;
}

}  // namespace gks

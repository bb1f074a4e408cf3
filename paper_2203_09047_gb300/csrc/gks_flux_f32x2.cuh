// FP32 Gauss-point flux (both forms, Eq. flux-1 and Eq. flux-2) with the two sides' work on
// packed f32x2 arithmetic: the flux templates are instantiated with the pair type P2, one
// half of every pair carrying the left side and the other the right. The per-side part --
// rotation of the reconstructed values and gradients into the face frame, primitives, the
// half-line moments rho <psi>_{u>0} and rho <psi>_{u<0} and their slopes along the three local
// axes, and for the full form the half-line fluxes F+, their second-moment and time-slope
// terms -- is the same arithmetic on both sides: about two thirds of the smooth form's
// operations and more of the full form's. The interface part (Q0, dW_d, the equilibrium terms,
// the time-fit weights) stays scalar and is shared with the scalar instantiation.
#pragma once
#include "gks_f32x2.cuh"
#include "gks_kinetic.cuh"

namespace gks {

// Both sides' values and gradients rotated into the face frame (as gp_flux_global).
__device__ __forceinline__ void rotate_in2(const float vl[5], const float gl[5][3],
                                           const float vr[5], const float gr[5][3],
                                           const float* const nm[3], P2 q[5], P2 dq[3][5]) {
  P2 N[3][3];
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int a = 0; a < 3; ++a) N[d][a] = P2(nm[d][a]);
  P2 V[5], G[5][3];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    V[v] = P2(vl[v], vr[v]);
#pragma unroll
    for (int a = 0; a < 3; ++a) G[v][a] = P2(gl[v][a], gr[v][a]);
  }
  q[0] = V[0];
  q[4] = V[4];
#pragma unroll
  for (int d = 0; d < 3; ++d) q[1 + d] = V[1] * N[d][0] + V[2] * N[d][1] + V[3] * N[d][2];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    P2 sd[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) sd[v] = G[v][0] * N[d][0] + G[v][1] * N[d][1] + G[v][2] * N[d][2];
    dq[d][0] = sd[0];
    dq[d][4] = sd[4];
#pragma unroll
    for (int e = 0; e < 3; ++e) dq[d][1 + e] = sd[1] * N[e][0] + sd[2] * N[e][1] + sd[3] * N[e][2];
  }
}

// Whole Gauss-point contribution in the global frame (as gp_flux_global): acc[0..4] = w F^n,
// acc[5..9] = w dF/dt. Returns false for a non-physical side or interface state.
__device__ __forceinline__ bool gp_flux_global2(const FluxParams<float>& P, const float vl[5],
                                                const float gl[5][3], const float vr[5],
                                                const float gr[5][3], const float n1[3],
                                                float w, float dt, float acc[10]) {
  P2 q[5], dq[3][5];
  float n2[3], n3[3];
  face_frame(n1, n2, n3);
  {
    const float* const nm[3] = {n1, n2, n3};
    rotate_in2(vl, gl, vr, gr, nm, q, dq);
  }
  const P2 gm1(P.gamma - 1.f), K2(P.K), sg(1.f, -1.f);  // sg: u > 0 left, u < 0 right
  Prim<P2> ws;
  if (!to_prim(q, P2(P.gamma), ws)) return false;
  Half<P2> hs;
  half_init(ws, K2, sg, hs);
  // interface equilibrium Q0 and its slopes dW_d: sums of the two half-line parts
  float q0[5], dW[3][5];
  {
    P2 Q[5];
    half_moments(ws, hs, Q);
#pragma unroll
    for (int v = 0; v < 5; ++v) q0[v] = hsum(Q[v]);
  }
  // the smooth form holds fewer values through the slopes with the interface primitives
  // formed after them and the frame formed again at the end (measured: 0.438 against 0.442 ms
  // per launch on the 64^3-cube mesh); the full form runs faster as written first (6.53
  // against 6.61 ms on the 128^3-cube explosion)
  Prim<float> w0;
  if (P.full && !to_prim(q0, P.gamma, w0)) return false;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    P2 t[5];
    half_jvp(ws, gm1, K2, sg, hs, dq[d], t);
#pragma unroll
    for (int v = 0; v < 5; ++v) dW[d][v] = hsum(t[v]);
  }
  if (!P.full && !to_prim(q0, P.gamma, w0)) return false;
  float dWt[5], E0[5], E1[5], E2[5], tau, Fn[5], Ft[5];
  interface_terms(P, ws.p.lo(), ws.p.hi(), q0, w0, dW, dt, dWt, E0, E1, E2, tau);
  if (!P.full) {
    smooth_from_terms(P, q0, w0, dWt, E0, E1, E2, tau, Fn, Ft);
  } else {
    // full form: both sides' non-equilibrium parts N0 = F+(W), N1 = sum_d DT+_d[dq_d],
    // N2 = DF+[rho <A psi>] with rho <A psi> = -sum_d A_d(W) dq_d (as gks_gp_flux)
    HalfLine<P2> ms;
    half_line(ws, hs, ms);
    P2 N[3][5], dts[5], t[5];
    half_flux(ws, K2, ms, N[0]);
    const P2 Ep = q[4] + ws.p;
    euler_jvp(ws, ws.ir, gm1, Ep, 0, dq[0], dts);
    half_second_jvp(ws, gm1, K2, sg, ms, 0, dq[0], N[1]);
#pragma unroll
    for (int d = 1; d < 3; ++d) {
      euler_jvp(ws, ws.ir, gm1, Ep, d, dq[d], t);
#pragma unroll
      for (int v = 0; v < 5; ++v) dts[v] += t[v];
      half_second_jvp(ws, gm1, K2, sg, ms, d, dq[d], t);
#pragma unroll
      for (int v = 0; v < 5; ++v) N[1][v] += t[v];
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) dts[v] = -dts[v];
    half_flux_jvp(ws, gm1, K2, sg, ms, dts, N[2]);
    float cn[6], ct[6];
    full_fit_coeffs(tau, dt, cn, ct);
    const P2 cn3(cn[3]), cn4(cn[4]), cn5(cn[5]), ct3(ct[3]), ct4(ct[4]), ct5(ct[5]);
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const P2 sn = cn3 * N[0][v] + cn4 * N[1][v] + cn5 * N[2][v];
      const P2 st = ct3 * N[0][v] + ct4 * N[1][v] + ct5 * N[2][v];
      Fn[v] = cn[0] * E0[v] + cn[1] * E1[v] + cn[2] * E2[v] + hsum(sn);
      Ft[v] = ct[0] * E0[v] + ct[1] * E1[v] + ct[2] * E2[v] + hsum(st);
    }
  }
  if (!P.full) face_frame(n1, n2, n3);
  rotate_flux_out(Fn, Ft, n1, n2, n3, w, acc);
  return true;
}

}  // namespace gks

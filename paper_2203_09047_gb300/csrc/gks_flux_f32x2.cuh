// FP32 smooth-form Gauss-point flux (Eq. flux-2) with the two sides' work on packed f32x2
// arithmetic (Blackwell FFMA2 / FMUL2 / FADD2: two FP32 operations per instruction and
// lane): one half of every pair carries the left side, the other the right. The per-side part
// of the flux -- rotation of the reconstructed value and gradients into the face frame, the
// primitives, the half-line moments rho <psi>_{u>0} and rho <psi>_{u<0}, and their derivatives
// along the three local axes -- is the same arithmetic on both sides, and it is about two
// thirds of the flux's operations. The interface part (Q0, dW_d and what follows) stays scalar
// and is shared with the scalar path (interface_terms, smooth_from_terms). Special functions
// and divisions run per half. The formulas are those of to_prim, half_init, half_moments and
// half_jvp, written out with explicit fused multiply-adds (the packed intrinsics are not
// contracted by the compiler).
#pragma once
#include "gks_kinetic.cuh"

namespace gks {

struct F2 {
  float2 v;
};
__device__ __forceinline__ F2 f2(float a, float b) { return {make_float2(a, b)}; }
__device__ __forceinline__ F2 bc(float a) { return {make_float2(a, a)}; }
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return {__fadd2_rn(a.v, b.v)}; }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return {__fmul2_rn(a.v, b.v)}; }
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) { return {__ffma2_rn(a.v, b.v, c.v)}; }
__device__ __forceinline__ float hsum(F2 a) { return a.v.x + a.v.y; }

// Both sides' primitives, half-line moments and the products their slopes reuse.
struct Side2 {
  F2 rho, U, V, W, p, lam, ir, ip, hil;  // as Prim
  F2 A, A1, A2, B, S;                    // as Half (s = +1 left, -1 right)
  // reused by the slopes
  F2 hu2, tl, tlU, Uh, sB, nA, nhK, VA, WA, hrho, hA2S;
};

// Primitives and half-line moments of both sides from their conserved states q (local frame).
// Returns false if either side has rho <= 0 or p <= 0 (or NaN).
__device__ __forceinline__ bool side2_init(const F2 q[5], float gamma, float K, Side2& s) {
  const F2 sg = f2(1.f, -1.f);
  s.rho = q[0];
  s.ir = f2(1.f / q[0].v.x, 1.f / q[0].v.y);
  s.U = q[1] * s.ir;
  s.V = q[2] * s.ir;
  s.W = q[3] * s.ir;
  const F2 mU = fma2(q[3], s.W, fma2(q[2], s.V, q[1] * s.U));
  s.p = bc(gamma - 1.f) * fma2(mU, bc(-0.5f), q[4]);
  s.ip = f2(1.f / s.p.v.x, 1.f / s.p.v.y);
  s.hrho = bc(0.5f) * s.rho;
  s.lam = s.hrho * s.ip;
  s.hil = s.p * s.ir;
  const bool ok = (s.rho.v.x > 0.f) && (s.rho.v.y > 0.f) && (s.p.v.x > 0.f) && (s.p.v.y > 0.f);
  // half lines u > 0 (left) and u < 0 (right)
  const F2 sl = f2(sqrtf(s.lam.v.x), sqrtf(s.lam.v.y));
  const F2 t = sl * s.U;
  s.A = bc(0.5f) * f2(erfcf(-t.v.x), erfcf(t.v.y));
  const F2 e = s.lam * s.U * s.U;
  s.B = bc(0.28209479177387814f) * f2(expf(-e.v.x) / sl.v.x, expf(-e.v.y) / sl.v.y);
  s.sB = sg * s.B;
  s.A1 = fma2(s.U, s.A, s.sB);
  s.A2 = fma2(s.U, s.A1, s.hil * s.A);
  const F2 K2hil = bc(K + 2.f) * s.hil;
  s.S = fma2(s.V, s.V, fma2(s.W, s.W, K2hil));
  // products reused by the three slopes
  const F2 m1 = bc(-1.f);
  s.hu2 = bc(0.5f) * fma2(s.U, s.U, fma2(s.V, s.V, s.W * s.W));
  s.tl = bc(2.f) * s.lam;
  s.tlU = s.tl * s.U;
  s.Uh = fma2(s.U, s.U, s.hil);
  s.nA = s.A * m1;
  s.nhK = K2hil * m1;
  s.VA = s.V * s.A;
  s.WA = s.W * s.A;
  s.hA2S = bc(0.5f) * fma2(s.S, s.A, s.A2);
  return ok;
}

// rho <psi> over each side's half line (as half_moments).
__device__ __forceinline__ void side2_moments(const Side2& s, F2 Q[5]) {
  Q[0] = s.rho * s.A;
  Q[1] = s.rho * s.A1;
  Q[2] = s.rho * s.VA;
  Q[3] = s.rho * s.WA;
  Q[4] = s.rho * s.hA2S;
}

// Derivative of both sides' half-line moments along their conserved increments dq (as
// half_jvp: dU = (dm - U drho)/rho, dp = (gamma - 1)(dE - U . dm + |U|^2 drho / 2),
// dlam/lam = drho/rho - dp/p, dA = s B (2 lam dU + U dlam), dB = -B (2 lam U dU + (U^2 +
// 1/(2 lam)) dlam), then the moment increments).
// gm1 = gamma - 1 in both halves.
__device__ __forceinline__ void side2_jvp(const Side2& s, F2 gm1, const F2 dq[5], F2 dQ[5]) {
  const F2 nsg = f2(-1.f, 1.f);  // -s: the sign of the half line, negated
  const F2 ndq0 = dq[0] * bc(-1.f);
  const F2 dU = fma2(s.U, ndq0, dq[1]) * s.ir;
  const F2 dV = fma2(s.V, ndq0, dq[2]) * s.ir;
  const F2 dW = fma2(s.W, ndq0, dq[3]) * s.ir;
  // t = -dp / (gamma - 1) = U . dm - dE - |U|^2 drho / 2, so that
  // dlam / lam = drho / rho - dp / p = drho / rho + (gamma - 1) t / p
  const F2 um = fma2(s.W, dq[3], fma2(s.V, dq[2], s.U * dq[1]));
  const F2 t = fma2(s.hu2, ndq0, um + dq[4] * bc(-1.f));
  const F2 dll = fma2(gm1 * t, s.ip, dq[0] * s.ir);
  const F2 dlam = s.lam * dll;
  const F2 dA = s.sB * fma2(s.tl, dU, s.U * dlam);
  const F2 mdB = s.B * fma2(s.tlU, dU, s.Uh * dlam);  // -dB
  const F2 dA1 = fma2(dU, s.A, fma2(s.U, dA, nsg * mdB));
  const F2 dA2 = fma2(dU, s.A1, fma2(s.U, dA1, s.hil * fma2(s.nA, dll, dA)));
  const F2 dS = fma2(bc(2.f), fma2(s.V, dV, s.W * dW), s.nhK * dll);
  dQ[0] = fma2(dq[0], s.A, s.rho * dA);
  dQ[1] = fma2(dq[0], s.A1, s.rho * dA1);
  dQ[2] = fma2(dq[0], s.VA, s.rho * fma2(dV, s.A, s.V * dA));
  dQ[3] = fma2(dq[0], s.WA, s.rho * fma2(dW, s.A, s.W * dA));
  dQ[4] = fma2(dq[0], s.hA2S, s.hrho * fma2(dS, s.A, fma2(s.S, dA, dA2)));
}

// Whole Gauss-point contribution of the smooth flux in the global frame (as gp_flux_global
// with P.full = 0): acc[0..4] = w F^n, acc[5..9] = w dF/dt. Returns false for a non-physical
// side or interface state.
__device__ __forceinline__ bool gp_flux_global_smooth2(const FluxParams<float>& P,
                                                       const float vl[5], const float gl[5][3],
                                                       const float vr[5], const float gr[5][3],
                                                       const float n1[3], float w, float dt,
                                                       float acc[10]) {
  float n2[3], n3[3];
  face_frame(n1, n2, n3);
  const float* nm[3] = {n1, n2, n3};
  F2 N[3][3];
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int a = 0; a < 3; ++a) N[d][a] = bc(nm[d][a]);
  // both sides' values and gradients, rotated into the face frame
  F2 V[5], G[5][3];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    V[v] = f2(vl[v], vr[v]);
#pragma unroll
    for (int a = 0; a < 3; ++a) G[v][a] = f2(gl[v][a], gr[v][a]);
  }
  F2 q[5], dq[3][5];
  q[0] = V[0];
  q[4] = V[4];
#pragma unroll
  for (int d = 0; d < 3; ++d)
    q[1 + d] = fma2(V[3], N[d][2], fma2(V[2], N[d][1], V[1] * N[d][0]));
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    F2 sd[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) sd[v] = fma2(G[v][2], N[d][2], fma2(G[v][1], N[d][1], G[v][0] * N[d][0]));
    dq[d][0] = sd[0];
    dq[d][4] = sd[4];
#pragma unroll
    for (int e = 0; e < 3; ++e)
      dq[d][1 + e] = fma2(sd[3], N[e][2], fma2(sd[2], N[e][1], sd[1] * N[e][0]));
  }
  Side2 s;
  if (!side2_init(q, P.gamma, P.K, s)) return false;
  // interface equilibrium Q0 and its slopes dW_d: sums of the two half-line parts
  float q0[5], dW[3][5];
  {
    F2 Q[5];
    side2_moments(s, Q);
#pragma unroll
    for (int v = 0; v < 5; ++v) q0[v] = hsum(Q[v]);
  }
  Prim<float> w0;
  if (!to_prim(q0, P.gamma, w0)) return false;
  const F2 gm1 = bc(P.gamma - 1.f);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    F2 dQ[5];
    side2_jvp(s, gm1, dq[d], dQ);
#pragma unroll
    for (int v = 0; v < 5; ++v) dW[d][v] = hsum(dQ[v]);
  }
  float dWt[5], E0[5], E1[5], E2[5], tau, Fn[5], Ft[5];
  interface_terms(P, s.p.v.x, s.p.v.y, q0, w0, dW, dt, dWt, E0, E1, E2, tau);
  smooth_from_terms(P, q0, w0, dWt, E0, E1, E2, tau, Fn, Ft);
  rotate_flux_out(Fn, Ft, n1, n2, n3, w, acc);
  return true;
}

}  // namespace gks

// Reverse of the closed-form Gauss-point flux of gks_kinetic.cuh, built from the structure of
// that forward code. Every term of the forward is either a function f(W) of a conserved state
// (the half-space moments, the Euler flux along an axis, the second-moment flux, the half-line
// flux and second-moment flux) or its derivative along an increment, J_f(W) x (the slopes of
// Eq. flux-1 and flux-2 written as directional derivatives). For the cotangent g of a term
// J_f(W) x the reverse needs J_f(W)^T g (the cotangent of x) and grad_W (g . J_f(W) x), the
// derivative of J_f(W)^T g along x (the cotangent of W). Both come from one evaluation of the
// hand-written reverse of the base function f, run in forward-mode dual numbers with W seeded
// along x: the value part is J_f(W)^T g, the tangent part its derivative along x. Only the six
// base functions need a hand-written reverse; no moment tables are kept.
#pragma once

#include "gks_kinetic.cuh"

namespace gks {

// Forward-mode dual number: value and one directional derivative.
template <class T>
struct Dl {
  T v, d;
  GKS_HD Dl() : v(T(0)), d(T(0)) {}
  GKS_HD Dl(T x) : v(x), d(T(0)) {}
  GKS_HD Dl(T x, T y) : v(x), d(y) {}
  GKS_HD explicit Dl(int x) : v(T(x)), d(T(0)) {}
};
template <class T> GKS_HD Dl<T> operator+(Dl<T> a, Dl<T> b) { return {a.v + b.v, a.d + b.d}; }
template <class T> GKS_HD Dl<T> operator-(Dl<T> a, Dl<T> b) { return {a.v - b.v, a.d - b.d}; }
template <class T> GKS_HD Dl<T> operator-(Dl<T> a) { return {-a.v, -a.d}; }
template <class T> GKS_HD Dl<T> operator*(Dl<T> a, Dl<T> b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
template <class T> GKS_HD Dl<T> operator/(Dl<T> a, Dl<T> b) {
  const T q = a.v / b.v;
  return {q, (a.d - q * b.d) / b.v};
}
template <class T> GKS_HD Dl<T>& operator+=(Dl<T>& a, Dl<T> b) { a = a + b; return a; }
template <class T> GKS_HD Dl<T>& operator-=(Dl<T>& a, Dl<T> b) { a = a - b; return a; }
template <class T> GKS_HD Dl<T>& operator*=(Dl<T>& a, Dl<T> b) { a = a * b; return a; }
template <class T> GKS_HD bool operator>(Dl<T> a, Dl<T> b) { return a.v > b.v; }
template <class T> GKS_HD bool operator<(Dl<T> a, Dl<T> b) { return a.v < b.v; }
GKS_HD Dl<double> k_exp(Dl<double> a) {
  const double e = exp(a.v);
  return {e, e * a.d};
}
GKS_HD Dl<double> k_sqrt(Dl<double> a) {
  const double s = sqrt(a.v);
  return {s, a.d / (2.0 * s)};
}
// d erfc(x)/dx = -(2 / sqrt(pi)) exp(-x^2)
GKS_HD Dl<double> k_erfc(Dl<double> a) {
  return {erfc(a.v), -1.1283791670955126 * exp(-a.v * a.v) * a.d};
}

// Reverse of to_prim: cotangents of (rho, U, V, W, p, lam, hil) -> those of the conserved state
// q (accumulated). lam = rho / (2 p), hil = p / rho, p = (gamma - 1) (E - |m|^2 / (2 rho)).
template <class R>
GKS_HD void prim_adj(const Prim<R>& w, R gm1, R gr, R gU, R gV, R gW, R gp, R glam, R ghil,
                     R gq[5]) {
  gr = gr + glam * R(0.5) * w.ip - ghil * w.hil * w.ir;
  gp = gp - glam * w.lam * w.ip + ghil * w.ir;
  const R gpe = gm1 * gp;
  gq[4] += gpe;
  gq[1] += gU * w.ir - gpe * w.U;
  gq[2] += gV * w.ir - gpe * w.V;
  gq[3] += gW * w.ir - gpe * w.W;
  gq[0] += gr + gpe * R(0.5) * (w.U * w.U + w.V * w.V + w.W * w.W) -
           (gU * w.U + gV * w.V + gW * w.W) * w.ir;
}

// Euler flux along axis d: F[0] = m_d, F[1 + a] = m_d U_a + p delta_ad, F[4] = U_d (E + p).
template <class R>
GKS_HD void euler_flux_vjp(const R q[5], R gamma, int d, const R g[5], R gq[5]) {
  Prim<R> w;
  to_prim(q, gamma, w);
  const R U[3] = {w.U, w.V, w.W};
  R gU[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) gU[a] = g[1 + a] * q[1 + d];
  gU[d] += g[4] * (q[4] + w.p);
  const R gp = g[1 + d] + g[4] * U[d];
  gq[1 + d] += g[0] + g[1] * U[0] + g[2] * U[1] + g[3] * U[2];
  gq[4] += g[4] * U[d];
  prim_adj(w, gamma - R(1), R(0), gU[0], gU[1], gU[2], gp, R(0), R(0), gq);
}

// Second-moment flux T_d(W) = rho <u c_d psi> (theta = p/rho, n = delta_0d):
//   t[0] = U_0 U_d + theta n, t[1 + a] = U_0 U_d U_a + theta (U_0 delta_da + U_d delta_0a + U_a n),
//   t[4] = (U_0 U_d (|U|^2 + (K + 7) theta) + n theta (|U|^2 + (K + 5) theta)) / 2, T = rho t.
template <class R>
GKS_HD void second_flux_vjp(const R q[5], R gamma, R K, int d, const R g[5], R gq[5]) {
  Prim<R> w;
  to_prim(q, gamma, w);
  const R U[3] = {w.U, w.V, w.W};
  const R th = w.hil, n = d == 0 ? R(1) : R(0);
  const R uu = U[0] * U[d], q2 = U[0] * U[0] + U[1] * U[1] + U[2] * U[2];
  const R c7 = K + R(7), c5 = K + R(5);
  R t[5];
  t[0] = uu + th * n;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const R ga = (a == d ? U[0] : R(0)) + (a == 0 ? U[d] : R(0)) + U[a] * n;
    t[1 + a] = uu * U[a] + th * ga;
  }
  t[4] = R(0.5) * (uu * (q2 + c7 * th) + n * th * (q2 + c5 * th));
  R gr = R(0);
#pragma unroll
  for (int k = 0; k < 5; ++k) gr += g[k] * t[k];
  R gt[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) gt[k] = w.rho * g[k];
  R guu = gt[0], gth = gt[0] * n, gq2 = R(0);
  R gU[3] = {R(0), R(0), R(0)};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const R ga = (a == d ? U[0] : R(0)) + (a == 0 ? U[d] : R(0)) + U[a] * n;
    guu += gt[1 + a] * U[a];
    gU[a] += gt[1 + a] * uu + gt[1 + a] * th * n;
    gth += gt[1 + a] * ga;
    if (a == d) gU[0] += gt[1 + a] * th;
    if (a == 0) gU[d] += gt[1 + a] * th;
  }
  guu += R(0.5) * gt[4] * (q2 + c7 * th);
  gq2 += R(0.5) * gt[4] * (uu + n * th);
  gth += R(0.5) * gt[4] * (uu * c7 + n * (q2 + R(2) * c5 * th));
  gU[0] += guu * U[d];
  gU[d] += guu * U[0];
#pragma unroll
  for (int a = 0; a < 3; ++a) gU[a] += R(2) * gq2 * U[a];
  prim_adj(w, gamma - R(1), gr, gU[0], gU[1], gU[2], R(0), R(0), gth, gq);
}

// Half-line moments of one side (s = +1: u > 0, s = -1: u < 0), as half_init and half_line:
// A0 = erfc(-s sqrt(lam) U) / 2, B = exp(-lam U^2) / (2 sqrt(pi lam)), A1 = U A0 + s B,
// A_{n+2} = U A_{n+1} + (n + 1) hil A_n. half_chain_adj turns the cotangents of A0..A4 and B
// into those of U, lam and hil (accumulated); dA0 = s B (2 lam dU + U dlam),
// dB = -B (2 lam U dU + (U^2 + 1/(2 lam)) dlam).
template <class R>
GKS_HD void half_chain(const Prim<R>& w, int s, R A[5], R& B) {
  const R sl = k_sqrt(w.lam);
  A[0] = R(0.5) * k_erfc(-R(s) * sl * w.U);
  B = R(0.28209479177387814) * k_exp(-w.lam * w.U * w.U) / sl;  // 1/(2 sqrt(pi))
  A[1] = w.U * A[0] + R(s) * B;
  A[2] = w.U * A[1] + w.hil * A[0];
  A[3] = w.U * A[2] + R(2) * w.hil * A[1];
  A[4] = w.U * A[3] + R(3) * w.hil * A[2];
}
template <class R>
GKS_HD void half_chain_adj(const Prim<R>& w, int s, const R A[5], R B, R gA[5], R gB, R& gU,
                           R& glam, R& ghil) {
  const R U = w.U, hil = w.hil;
  gA[3] += gA[4] * U;
  gU += gA[4] * A[3];
  ghil += R(3) * gA[4] * A[2];
  gA[2] += R(3) * gA[4] * hil;
  gA[2] += gA[3] * U;
  gU += gA[3] * A[2];
  ghil += R(2) * gA[3] * A[1];
  gA[1] += R(2) * gA[3] * hil;
  gA[1] += gA[2] * U;
  gU += gA[2] * A[1];
  ghil += gA[2] * A[0];
  gA[0] += gA[2] * hil;
  gA[0] += gA[1] * U;
  gU += gA[1] * A[0];
  gB += R(s) * gA[1];
  gU += (gA[0] * R(s) - gB * U) * R(2) * w.lam * B;
  glam += (gA[0] * R(s) * U - gB * (U * U + hil)) * B;
}

// Half-space conserved moments rho <psi>_s = rho (A0, A1, V A0, W A0, (A2 + S A0) / 2),
// S = V^2 + W^2 + (K + 2) hil.
template <class R>
GKS_HD void half_mom_vjp(const R q[5], R gamma, R K, int s, const R g[5], R gq[5]) {
  Prim<R> w;
  to_prim(q, gamma, w);
  R A[5], B;
  half_chain(w, s, A, B);
  const R S = w.V * w.V + w.W * w.W + (K + R(2)) * w.hil;
  const R gr = g[0] * A[0] + g[1] * A[1] + g[2] * w.V * A[0] + g[3] * w.W * A[0] +
               R(0.5) * g[4] * (A[2] + S * A[0]);
  R gA[5] = {w.rho * (g[0] + g[2] * w.V + g[3] * w.W + R(0.5) * g[4] * S), w.rho * g[1],
             R(0.5) * w.rho * g[4], R(0), R(0)};
  const R gS = R(0.5) * w.rho * g[4] * A[0];
  const R gV = w.rho * g[2] * A[0] + R(2) * w.V * gS, gW = w.rho * g[3] * A[0] + R(2) * w.W * gS;
  R gU = R(0), glam = R(0), ghil = (K + R(2)) * gS;
  half_chain_adj(w, s, A, B, gA, R(0), gU, glam, ghil);
  prim_adj(w, gamma - R(1), gr, gU, gV, gW, R(0), glam, ghil, gq);
}

// Half-line flux F_s(W) = rho <u psi>_s = rho (A1, A2, V A1, W A1, (A3 + S A1) / 2).
template <class R>
GKS_HD void half_flux_vjp(const R q[5], R gamma, R K, int s, const R g[5], R gq[5]) {
  Prim<R> w;
  to_prim(q, gamma, w);
  R A[5], B;
  half_chain(w, s, A, B);
  const R S = w.V * w.V + w.W * w.W + (K + R(2)) * w.hil;
  const R gr = g[0] * A[1] + g[1] * A[2] + g[2] * w.V * A[1] + g[3] * w.W * A[1] +
               R(0.5) * g[4] * (A[3] + S * A[1]);
  R gA[5] = {R(0), w.rho * (g[0] + g[2] * w.V + g[3] * w.W + R(0.5) * g[4] * S), w.rho * g[1],
             R(0.5) * w.rho * g[4], R(0)};
  const R gS = R(0.5) * w.rho * g[4] * A[1];
  const R gV = w.rho * g[2] * A[1] + R(2) * w.V * gS, gW = w.rho * g[3] * A[1] + R(2) * w.W * gS;
  R gU = R(0), glam = R(0), ghil = (K + R(2)) * gS;
  half_chain_adj(w, s, A, B, gA, R(0), gU, glam, ghil);
  prim_adj(w, gamma - R(1), gr, gU, gV, gW, R(0), glam, ghil, gq);
}

// Half-line second-moment flux T_s,k(W) = rho <u c_k psi>_s (k = 0 normal, 1, 2 tangential):
//   k = 0: rho (A2, A3, V A2, W A2, (A4 + S A2) / 2);
//   k = 1, 2 with c the component k and o the other one: rho (c A1, c A2, [c^2 + hil] A1 at c's
//   slot, c o A1 at o's slot, (c A3 + c (V^2 + W^2 + (K + 4) hil) A1) / 2).
template <class R>
GKS_HD void half_second_vjp(const R q[5], R gamma, R K, int s, int k, const R g[5], R gq[5]) {
  Prim<R> w;
  to_prim(q, gamma, w);
  R A[5], B;
  half_chain(w, s, A, B);
  R gA[5] = {R(0), R(0), R(0), R(0), R(0)};
  R gr, gV = R(0), gW = R(0), ghil = R(0);
  if (k == 0) {
    const R S = w.V * w.V + w.W * w.W + (K + R(2)) * w.hil;
    gr = g[0] * A[2] + g[1] * A[3] + g[2] * w.V * A[2] + g[3] * w.W * A[2] +
         R(0.5) * g[4] * (A[4] + S * A[2]);
    gA[2] = w.rho * (g[0] + g[2] * w.V + g[3] * w.W + R(0.5) * g[4] * S);
    gA[3] = w.rho * g[1];
    gA[4] = R(0.5) * w.rho * g[4];
    const R gS = R(0.5) * w.rho * g[4] * A[2];
    gV = w.rho * g[2] * A[2] + R(2) * w.V * gS;
    gW = w.rho * g[3] * A[2] + R(2) * w.W * gS;
    ghil = (K + R(2)) * gS;
  } else {
    const R c = k == 1 ? w.V : w.W, o = k == 1 ? w.W : w.V;
    const R gcs = k == 1 ? g[2] : g[3], gos = k == 1 ? g[3] : g[2];  // c's and o's slots
    const R c2 = c * c + w.hil;
    const R qq = w.V * w.V + w.W * w.W + (K + R(4)) * w.hil;
    const R Y = c * qq;
    gr = g[0] * c * A[1] + g[1] * c * A[2] + gcs * c2 * A[1] + gos * c * o * A[1] +
         R(0.5) * g[4] * (c * A[3] + Y * A[1]);
    const R r0 = w.rho * g[0], r1 = w.rho * g[1], rc = w.rho * gcs, ro = w.rho * gos,
            r4 = w.rho * g[4];
    const R gc = r0 * A[1] + r1 * A[2] + rc * R(2) * c * A[1] + ro * o * A[1] +
                 R(0.5) * r4 * (A[3] + qq * A[1]);
    const R go = ro * c * A[1];
    const R gqq = R(0.5) * r4 * c * A[1];
    ghil = rc * A[1] + (K + R(4)) * gqq;
    gA[1] = r0 * c + rc * c2 + ro * c * o + R(0.5) * r4 * Y;
    gA[2] = r1 * c;
    gA[3] = R(0.5) * r4 * c;
    gV = R(2) * w.V * gqq + (k == 1 ? gc : go);
    gW = R(2) * w.W * gqq + (k == 1 ? go : gc);
  }
  R gU = R(0), glam = R(0);
  half_chain_adj(w, s, A, B, gA, R(0), gU, glam, ghil);
  prim_adj(w, gamma - R(1), gr, gU, gV, gW, R(0), glam, ghil, gq);
}

// Base functions by kind (for the dual-number evaluations below).
enum : int { kBaseHalfMom = 0, kBaseEuler = 1, kBaseSecond = 2, kBaseHalfFlux = 3, kBaseHalfSecond = 4 };
template <class R>
GKS_HD void base_vjp(int kind, int s, int k, const R q[5], R gamma, R K, const R g[5], R gq[5]) {
  switch (kind) {
    case kBaseHalfMom: half_mom_vjp(q, gamma, K, s, g, gq); break;
    case kBaseEuler: euler_flux_vjp(q, gamma, k, g, gq); break;
    case kBaseSecond: second_flux_vjp(q, gamma, K, k, g, gq); break;
    case kBaseHalfFlux: half_flux_vjp(q, gamma, K, s, g, gq); break;
    default: half_second_vjp(q, gamma, K, s, k, g, gq); break;
  }
}
// For the term J_f(q) x with cotangent g: gx += J_f(q)^T g and gq += grad_q (g . J_f(q) x).
GKS_HD void term_vjp(int kind, int s, int k, const double q[5], const double x[5],
                            const double g[5], double gamma, double K, double gx[5],
                            double gq[5]) {
  Dl<double> qd[5], gd[5], out[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    qd[v] = Dl<double>(q[v], x[v]);
    gd[v] = Dl<double>(g[v]);
  }
  base_vjp(kind, s, k, qd, Dl<double>(gamma), Dl<double>(K), gd, out);
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    gx[v] += out[v].v;
    gq[v] += out[v].d;
  }
}

// d/dtau of the six time integrals of Eq. flux-1 over [0, d] (flux1_integrals).
GKS_HD void flux1_dtau(double tau, double d, double dc[6]) {
  const double e = exp(-d / tau), om = 1.0 - e, r = d / tau;
  const double de = e * r / tau;  // d e / d tau
  dc[0] = -om + tau * de;
  dc[1] = 4.0 * tau * om - 2.0 * tau * tau * de - d * (1.0 + e) - tau * d * de;
  dc[2] = -d + 2.0 * tau * om - tau * tau * de;
  dc[3] = om - tau * de;
  dc[4] = d * e + tau * d * de - 4.0 * tau * om + 2.0 * tau * tau * de;
  dc[5] = -2.0 * tau * om + tau * tau * de;
}

// Vector-Jacobian product of gks_gp_flux (FP64): cotangents gFn, gFt of (F^n, dF/dt) ->
// cotangents of ql, dql, qr, dqr (accumulated). The forward is recomputed with the forward's own
// helpers; the reverse walks it backwards term by term. Returns false for a non-physical state.
// The heat-flux correction (Pr != 1) is not reversed.
GKS_HD bool gks_gp_flux_vjp_cf(const FluxParams<double>& P, const double ql[5],
                                      const double dql[3][5], const double qr[5],
                                      const double dqr[3][5], double dt, const double gFn[5],
                                      const double gFt[5], double gql[5], double gdql[3][5],
                                      double gqr[5], double gdqr[3][5]) {
  typedef double R;
  // ---- forward
  Prim<R> wl, wr, w0;
  if (!(to_prim(ql, P.gamma, wl) & to_prim(qr, P.gamma, wr))) return false;
  const R gm1 = P.gamma - R(1), K = P.K;
  Half<R> hl, hr;
  half_init(wl, K, +1, hl);
  half_init(wr, K, -1, hr);
  R q0[5], t[5];
  half_moments(wl, hl, q0);
  half_moments(wr, hr, t);
#pragma unroll
  for (int q = 0; q < 5; ++q) q0[q] += t[q];
  if (!to_prim(q0, P.gamma, w0)) return false;
  R dW[3][5];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    half_jvp(wl, gm1, K, +1, hl, dql[d], dW[d]);
    half_jvp(wr, gm1, K, -1, hr, dqr[d], t);
#pragma unroll
    for (int q = 0; q < 5; ++q) dW[d][q] += t[q];
  }
  const R ir0 = w0.ir, Ep0 = q0[4] + w0.p;
  R dWt[5], E0[5], E1[5] = {R(0), R(0), R(0), R(0), R(0)}, E2[5];
  euler_jvp(w0, ir0, gm1, Ep0, 0, dW[0], dWt);
#pragma unroll
  for (int d = 1; d < 3; ++d) {
    euler_jvp(w0, ir0, gm1, Ep0, d, dW[d], t);
#pragma unroll
    for (int q = 0; q < 5; ++q) dWt[q] += t[q];
  }
#pragma unroll
  for (int q = 0; q < 5; ++q) dWt[q] = -dWt[q];
  euler_flux_x(w0, q0[4], E0);
  euler_jvp(w0, ir0, gm1, Ep0, 0, dWt, E2);
  const R sdp = wl.p >= wr.p ? R(1) : R(-1), spp = wl.p + wr.p;
  const R dp = sdp * (wl.p - wr.p) / spp;
  const R tau = collision_time(P, w0.p, ir0, dp, dt);
  if (P.tau_model != 0) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      second_moment_jvp(w0, ir0, gm1, K, d, dW[d], t);
#pragma unroll
      for (int q = 0; q < 5; ++q) E1[q] += t[q];
    }
  }
  // ---- reverse of the combination
  R gE0[5], gE1[5], gE2[5], gtau = R(0);
  R gdW[3][5], gq0[5] = {R(0), R(0), R(0), R(0), R(0)};
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int q = 0; q < 5; ++q) gdW[d][q] = R(0);
  if (!P.full) {
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      gE0[q] = gFn[q];
      gE1[q] = -tau * gFn[q];
      gE2[q] = gFt[q] - tau * gFn[q];
      gtau -= gFn[q] * (E1[q] + E2[q]);
    }
  } else {
    R cn[6], ct[6], dcn[6], dct[6];
    if (tau > R(0)) {
      R ch[6], cf[6], dch[6], dcf[6];
      flux1_integrals(tau, R(0.5) * dt, ch);
      flux1_integrals(tau, dt, cf);
      flux1_dtau(tau, R(0.5) * dt, dch);
      flux1_dtau(tau, dt, dcf);
      const R idt = R(1) / dt;
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        cn[q] = (R(4) * ch[q] - cf[q]) * idt;
        ct[q] = R(4) * (cf[q] - R(2) * ch[q]) * idt * idt;
        dcn[q] = (R(4) * dch[q] - dcf[q]) * idt;
        dct[q] = R(4) * (dcf[q] - R(2) * dch[q]) * idt * idt;
      }
    } else {
#pragma unroll
      for (int q = 0; q < 6; ++q) cn[q] = ct[q] = dcn[q] = dct[q] = R(0);
      cn[0] = R(1);
      ct[2] = R(1);
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      gE0[q] = cn[0] * gFn[q] + ct[0] * gFt[q];
      gE1[q] = cn[1] * gFn[q] + ct[1] * gFt[q];
      gE2[q] = cn[2] * gFn[q] + ct[2] * gFt[q];
      gtau += gFn[q] * (dcn[0] * E0[q] + dcn[1] * E1[q] + dcn[2] * E2[q]) +
              gFt[q] * (dct[0] * E0[q] + dct[1] * E1[q] + dct[2] * E2[q]);
    }
    // the non-equilibrium parts of both sides
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const int s = side == 0 ? 1 : -1;
      const R* qs = side == 0 ? ql : qr;
      const R (*dqs)[5] = side == 0 ? dql : dqr;
      R* gqs = side == 0 ? gql : gqr;
      R (*gdqs)[5] = side == 0 ? gdql : gdqr;
      Prim<R> ws;
      to_prim(qs, P.gamma, ws);
      Half<R> hs;
      half_init(ws, K, s, hs);
      HalfLine<R> ms;
      half_line(ws, hs, ms);
      R N[3][5], dts[5];
      half_flux(ws, K, ms, N[0]);
      const R Eps = qs[4] + ws.p;
      euler_jvp(ws, ws.ir, gm1, Eps, 0, dqs[0], dts);
#pragma unroll
      for (int d = 1; d < 3; ++d) {
        euler_jvp(ws, ws.ir, gm1, Eps, d, dqs[d], t);
#pragma unroll
        for (int q = 0; q < 5; ++q) dts[q] += t[q];
      }
#pragma unroll
      for (int q = 0; q < 5; ++q) dts[q] = -dts[q];
      half_second_jvp(ws, gm1, K, s, ms, 0, dqs[0], N[1]);
#pragma unroll
      for (int d = 1; d < 3; ++d) {
        half_second_jvp(ws, gm1, K, s, ms, d, dqs[d], t);
#pragma unroll
        for (int q = 0; q < 5; ++q) N[1][q] += t[q];
      }
      half_flux_jvp(ws, gm1, K, s, ms, dts, N[2]);
      R gN[3][5];
#pragma unroll
      for (int q = 0; q < 5; ++q) {
#pragma unroll
        for (int j = 0; j < 3; ++j) gN[j][q] = cn[3 + j] * gFn[q] + ct[3 + j] * gFt[q];
        gtau += gFn[q] * (dcn[3] * N[0][q] + dcn[4] * N[1][q] + dcn[5] * N[2][q]) +
                gFt[q] * (dct[3] * N[0][q] + dct[4] * N[1][q] + dct[5] * N[2][q]);
      }
      // N0 = F_s(q): gq += J^T gN0 (a plain reverse, no direction)
      base_vjp<R>(kBaseHalfFlux, s, 0, qs, P.gamma, K, gN[0], gqs);
      // N1 = sum_d T_s,d'(q)[dq_d]
#pragma unroll
      for (int d = 0; d < 3; ++d)
        term_vjp(kBaseHalfSecond, s, d, qs, dqs[d], gN[1], P.gamma, K, gdqs[d], gqs);
      // N2 = F_s'(q)[dts], dts = -sum_d A_d(q) dq_d
      R gdts[5] = {R(0), R(0), R(0), R(0), R(0)};
      term_vjp(kBaseHalfFlux, s, 0, qs, dts, gN[2], P.gamma, K, gdts, gqs);
      R mg[5];
#pragma unroll
      for (int q = 0; q < 5; ++q) mg[q] = -gdts[q];
#pragma unroll
      for (int d = 0; d < 3; ++d) term_vjp(kBaseEuler, 0, d, qs, dqs[d], mg, P.gamma, K, gdqs[d], gqs);
    }
  }
  // ---- reverse of the interface equilibrium terms
  // E2 = A_0(q0) dWt
  R gdWt[5] = {R(0), R(0), R(0), R(0), R(0)};
  term_vjp(kBaseEuler, 0, 0, q0, dWt, gE2, P.gamma, K, gdWt, gq0);
  // E0 = F_0(q0)
  base_vjp<R>(kBaseEuler, 0, 0, q0, P.gamma, K, gE0, gq0);
  // E1 = sum_d T_d'(q0)[dW_d]
  if (P.tau_model != 0)
#pragma unroll
    for (int d = 0; d < 3; ++d) term_vjp(kBaseSecond, 0, d, q0, dW[d], gE1, P.gamma, K, gdW[d], gq0);
  // dWt = -sum_d A_d(q0) dW_d
  R mg[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) mg[q] = -gdWt[q];
#pragma unroll
  for (int d = 0; d < 3; ++d) term_vjp(kBaseEuler, 0, d, q0, dW[d], mg, P.gamma, K, gdW[d], gq0);
  // collision time: tau(p0, rho0, dp), dp = |pl - pr| / (pl + pr) (d|x|/dx = sign, +1 at 0)
  if (P.tau_model != 0) {
    R gp0 = R(0), gr0 = R(0), gdp = R(0);
    if (P.tau_model == 1) {
      gdp = gtau * P.tau_C * dt;
    } else if (P.tau_model == 2) {
      gp0 = -gtau * P.mu / (w0.p * w0.p);
      gdp = gtau * P.tau_C * dt;
    } else {
      // mu (p0 / (rho0 T_ref))^mu_pow / p0 = mu T_ref^-mu_pow p0^(mu_pow - 1) rho0^-mu_pow
      const R a = P.mu * k_pow(w0.p * ir0 / P.T_ref, P.mu_pow) / w0.p;
      gp0 = gtau * a * (P.mu_pow - R(1)) / w0.p;
      gr0 = -gtau * a * P.mu_pow * ir0;
      gdp = gtau * P.tau_C * dt;
    }
    prim_adj(w0, gm1, gr0, R(0), R(0), R(0), gp0, R(0), R(0), gq0);
    // dp = sdp (pl - pr) / (pl + pr)
    const R gpl = gdp * (sdp - dp) / spp, gpr = gdp * (-sdp - dp) / spp;
    prim_adj(wl, gm1, R(0), R(0), R(0), R(0), gpl, R(0), R(0), gql);
    prim_adj(wr, gm1, R(0), R(0), R(0), R(0), gpr, R(0), R(0), gqr);
  }
  // dW_d = M_+'(ql)[dql_d] + M_-'(qr)[dqr_d]
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    term_vjp(kBaseHalfMom, +1, 0, ql, dql[d], gdW[d], P.gamma, K, gdql[d], gql);
    term_vjp(kBaseHalfMom, -1, 0, qr, dqr[d], gdW[d], P.gamma, K, gdqr[d], gqr);
  }
  // q0 = M_+(ql) + M_-(qr)
  base_vjp<R>(kBaseHalfMom, +1, 0, ql, P.gamma, K, gq0, gql);
  base_vjp<R>(kBaseHalfMom, -1, 0, qr, P.gamma, K, gq0, gqr);
  return true;
}

}  // namespace gks

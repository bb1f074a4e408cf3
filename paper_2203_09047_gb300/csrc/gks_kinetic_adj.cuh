// Reverse-mode (vector-Jacobian) companion of gks_kinetic.cuh: the adjoint of the Gauss-point
// gas-kinetic flux, written by hand step by step in the reverse order of the forward code.
// Forward intermediates are recomputed (no tape). Every helper mirrors one forward helper.
#pragma once

#include "gks_kinetic.cuh"

namespace gks {

template <class R>
GKS_HD void mom_zero(Mom<R>& g) {
#pragma unroll
  for (int k = 0; k < 7; ++k) g.u[k] = R(0);
#pragma unroll
  for (int k = 0; k < 6; ++k) g.v[k] = g.w[k] = R(0);
  g.xi[0] = g.xi[1] = g.xi[2] = R(0);
}

// Adjoint of one product term coef * u[a] v[b] w[c] xi[d] with cotangent g.
template <class R>
GKS_HD void term_adj(const Mom<R>& M, Mom<R>& gM, int a, int b, int c, int d, R cg) {
  gM.u[a] += cg * M.v[b] * M.w[c] * M.xi[d];
  gM.v[b] += cg * M.u[a] * M.w[c] * M.xi[d];
  gM.w[c] += cg * M.u[a] * M.v[b] * M.xi[d];
  gM.xi[d] += cg * M.u[a] * M.v[b] * M.w[c];
}

// Adjoint of G(M, k, l, m, x) with output cotangent g[5].
template <class R>
GKS_HD void G_adj(const Mom<R>& M, Mom<R>& gM, int k, int l, int m, int x, const R g[5]) {
  term_adj(M, gM, k, l, m, x, g[0]);
  term_adj(M, gM, k + 1, l, m, x, g[1]);
  term_adj(M, gM, k, l + 1, m, x, g[2]);
  term_adj(M, gM, k, l, m + 1, x, g[3]);
  const R h = R(0.5) * g[4];
  term_adj(M, gM, k + 2, l, m, x, h);
  term_adj(M, gM, k, l + 2, m, x, h);
  term_adj(M, gM, k, l, m + 2, x, h);
  term_adj(M, gM, k, l, m, x + 1, h);
}

// Adjoint of Ga(M, a, k, l, m): accumulates into gM and ga.
template <class R>
GKS_HD void Ga_adj(const Mom<R>& M, const R a[5], int k, int l, int m, const R g[5], Mom<R>& gM,
                   R ga[5]) {
  R t[5], s[5];
  G(M, k, l, m, 0, t);
  R d = R(0);
#pragma unroll
  for (int q = 0; q < 5; ++q) d += g[q] * t[q];
  ga[0] += d;
#pragma unroll
  for (int q = 0; q < 5; ++q) s[q] = a[0] * g[q];
  G_adj(M, gM, k, l, m, 0, s);
  G(M, k + 1, l, m, 0, t);
  d = R(0);
#pragma unroll
  for (int q = 0; q < 5; ++q) d += g[q] * t[q];
  ga[1] += d;
#pragma unroll
  for (int q = 0; q < 5; ++q) s[q] = a[1] * g[q];
  G_adj(M, gM, k + 1, l, m, 0, s);
  G(M, k, l + 1, m, 0, t);
  d = R(0);
#pragma unroll
  for (int q = 0; q < 5; ++q) d += g[q] * t[q];
  ga[2] += d;
#pragma unroll
  for (int q = 0; q < 5; ++q) s[q] = a[2] * g[q];
  G_adj(M, gM, k, l + 1, m, 0, s);
  G(M, k, l, m + 1, 0, t);
  d = R(0);
#pragma unroll
  for (int q = 0; q < 5; ++q) d += g[q] * t[q];
  ga[3] += d;
#pragma unroll
  for (int q = 0; q < 5; ++q) s[q] = a[3] * g[q];
  G_adj(M, gM, k, l, m + 1, 0, s);
  // a4/2 (G(k+2) + G(l+2) + G(m+2) + G(x+1))
  R sum[5];
  G(M, k + 2, l, m, 0, sum);
  G(M, k, l + 2, m, 0, t);
#pragma unroll
  for (int q = 0; q < 5; ++q) sum[q] += t[q];
  G(M, k, l, m + 2, 0, t);
#pragma unroll
  for (int q = 0; q < 5; ++q) sum[q] += t[q];
  G(M, k, l, m, 1, t);
#pragma unroll
  for (int q = 0; q < 5; ++q) sum[q] += t[q];
  d = R(0);
#pragma unroll
  for (int q = 0; q < 5; ++q) d += g[q] * sum[q];
  ga[4] += R(0.5) * d;
#pragma unroll
  for (int q = 0; q < 5; ++q) s[q] = R(0.5) * a[4] * g[q];
  G_adj(M, gM, k + 2, l, m, 0, s);
  G_adj(M, gM, k, l + 2, m, 0, s);
  G_adj(M, gM, k, l, m + 2, 0, s);
  G_adj(M, gM, k, l, m, 1, s);
}

template <class R>
GKS_HD void Gadotu_adj(const Mom<R>& M, const R a[3][5], int k, const R g[5], Mom<R>& gM,
                       R ga[3][5]) {
  Ga_adj(M, a[0], k + 1, 0, 0, g, gM, ga[0]);
  Ga_adj(M, a[1], k, 1, 0, g, gM, ga[1]);
  Ga_adj(M, a[2], k, 0, 1, g, gM, ga[2]);
}

// Adjoint of line_moments<N>(c, hil): accumulates into gc, ghil; consumes g (modified).
template <class R, int N>
GKS_HD void line_moments_adj(R c, R hil, const R* out, R* g, R& gc, R& ghil) {
  for (int n = N - 1; n >= 2; --n) {
    gc += g[n] * out[n - 1];
    g[n - 1] += g[n] * c;
    ghil += g[n] * R(n - 1) * out[n - 2];
    g[n - 2] += g[n] * R(n - 1) * hil;
  }
  gc += g[1];
}

// Adjoint of maxwell_moments: gM (consumed) -> gU, gV, gW, glam.
template <class R>
GKS_HD void maxwell_moments_adj(R U, R V, R W, R lam, R K, int side, const Mom<R>& M, Mom<R>& gM,
                                R& gU, R& gV, R& gW, R& glam) {
  const R hil = R(0.5) / lam;
  R ghil = R(0);
  ghil += gM.xi[1] * K + gM.xi[2] * R(2) * K * (K + R(2)) * hil;
  line_moments_adj<R, 6>(V, hil, M.v, gM.v, gV, ghil);
  line_moments_adj<R, 6>(W, hil, M.w, gM.w, gW, ghil);
  if (side == 0) {
    line_moments_adj<R, 7>(U, hil, M.u, gM.u, gU, ghil);
  } else {
    // recurrence part n >= 2
    for (int n = 6; n >= 2; --n) {
      gU += gM.u[n] * M.u[n - 1];
      gM.u[n - 1] += gM.u[n] * U;
      ghil += gM.u[n] * R(n - 1) * M.u[n - 2];
      gM.u[n - 2] += gM.u[n] * R(n - 1) * hil;
    }
    const R s = R(side);
    const R sl = k_sqrt(lam);
    const R e = k_exp(-lam * U * U);
    const R c = R(0.28209479177387814);  // 1/(2 sqrt(pi))
    // u1 = U u0 + s c e / sqrt(lam)
    gU += gM.u[1] * M.u[0];
    gM.u[0] += gM.u[1] * U;
    const R ge = gM.u[1] * s * c / sl;
    glam += gM.u[1] * s * c * e * (R(-0.5) / (lam * sl));
    glam += ge * e * (-U * U);
    gU += ge * e * (R(-2) * lam * U);
    // u0 = erfc(z) / 2, z = -s sqrt(lam) U; d erfc/dz = -2/sqrt(pi) exp(-z^2), exp(-z^2) = e
    const R gz = -gM.u[0] * e * R(0.5641895835477563);  // 1/sqrt(pi)
    gU += gz * (-s * sl);
    glam += gz * (-s * U * R(0.5) / sl);
  }
  glam += -ghil * R(0.5) / (lam * lam);
}

// Adjoint of slope_solve: ga (input cotangent of a) -> gU, gV, gW, glam, gb.
template <class R>
GKS_HD void slope_solve_adj(R U, R V, R W, R lam, R K, const R b[5], const R ga_in[5], R& gU,
                            R& gV, R& gW, R& glam, R gb[5]) {
  // forward recomputation
  const R q2 = U * U + V * V + W * W;
  const R e2 = q2 + (K + R(3)) * R(0.5) / lam;
  const R r1 = b[1] - U * b[0], r2 = b[2] - V * b[0], r3 = b[3] - W * b[0];
  const R r4 = R(2) * b[4] - e2 * b[0];
  const R cc = R(4) * lam * lam / (K + R(3));
  const R S = U * r1 + V * r2 + W * r3;
  const R a4 = cc * (r4 - R(2) * S);
  const R tl = R(2) * lam;
  const R a1 = tl * r1 - U * a4, a2 = tl * r2 - V * a4, a3 = tl * r3 - W * a4;
  // a0 = b0 - U a1 - V a2 - W a3 - a4 e2 / 2
  R ga1 = ga_in[1] - U * ga_in[0], ga2 = ga_in[2] - V * ga_in[0], ga3 = ga_in[3] - W * ga_in[0];
  R ga4 = ga_in[4] - R(0.5) * e2 * ga_in[0];
  R ge2 = -R(0.5) * a4 * ga_in[0];
  gU += -a1 * ga_in[0];
  gV += -a2 * ga_in[0];
  gW += -a3 * ga_in[0];
  gb[0] += ga_in[0];
  // a_i = tl r_i - U_i a4
  R gtl = r1 * ga1 + r2 * ga2 + r3 * ga3;
  R gr1 = tl * ga1, gr2 = tl * ga2, gr3 = tl * ga3;
  gU += -a4 * ga1;
  gV += -a4 * ga2;
  gW += -a4 * ga3;
  ga4 += -U * ga1 - V * ga2 - W * ga3;
  glam += R(2) * gtl;
  // a4 = cc (r4 - 2 S)
  glam += (r4 - R(2) * S) * ga4 * R(8) * lam / (K + R(3));
  const R gr4 = cc * ga4;
  const R gS = R(-2) * cc * ga4;
  gU += r1 * gS;
  gV += r2 * gS;
  gW += r3 * gS;
  gr1 += U * gS;
  gr2 += V * gS;
  gr3 += W * gS;
  // r4 = 2 b4 - e2 b0
  gb[4] += R(2) * gr4;
  ge2 += -b[0] * gr4;
  gb[0] += -e2 * gr4;
  // r_i = b_i - U_i b0
  gb[1] += gr1;
  gb[2] += gr2;
  gb[3] += gr3;
  gU += -b[0] * gr1;
  gV += -b[0] * gr2;
  gW += -b[0] * gr3;
  gb[0] += -U * gr1 - V * gr2 - W * gr3;
  // e2 = q2 + (K+3)/(2 lam)
  glam += ge2 * (-(K + R(3)) * R(0.5) / (lam * lam));
  gU += R(2) * U * ge2;
  gV += R(2) * V * ge2;
  gW += R(2) * W * ge2;
}

// Cotangents of a primitive state.
template <class R>
struct PrimAdj {
  R rho = R(0), U = R(0), V = R(0), W = R(0), p = R(0), lam = R(0);
};

// Adjoint of to_prim: g (consumed) -> gq[5] (accumulated).
template <class R>
GKS_HD void to_prim_adj(const R q[5], R gamma, const Prim<R>& w, const PrimAdj<R>& g, R gq[5]) {
  // lam = rho / (2 p)
  const R grho = g.rho + g.lam * R(0.5) / w.p;
  const R gp = g.p - g.lam * R(0.5) * w.rho / (w.p * w.p);
  // p = (gamma - 1) (q4 - (q1 U + q2 V + q3 W) / 2)
  const R gm1 = gamma - R(1);
  gq[4] += gm1 * gp;
  const R gUt = g.U - gm1 * R(0.5) * q[1] * gp;
  const R gVt = g.V - gm1 * R(0.5) * q[2] * gp;
  const R gWt = g.W - gm1 * R(0.5) * q[3] * gp;
  gq[1] += -gm1 * R(0.5) * w.U * gp;
  gq[2] += -gm1 * R(0.5) * w.V * gp;
  gq[3] += -gm1 * R(0.5) * w.W * gp;
  // U = q1 / q0 ...
  const R ir = R(1) / q[0];
  gq[1] += gUt * ir;
  gq[2] += gVt * ir;
  gq[3] += gWt * ir;
  gq[0] += -(gUt * w.U + gVt * w.V + gWt * w.W) * ir;
  gq[0] += grho;
}

// d/dtau of the six time integrals of Eq. flux-1 over [0, d].
template <class R>
GKS_HD void flux1_integrals_dtau(R tau, R d, R dc[6]) {
  const R e = k_exp(-d / tau);
  const R om = R(1) - e;
  const R de = e * d / (tau * tau);
  const R dom = -de;
  dc[0] = -om - tau * dom;
  dc[1] = R(4) * tau * om + R(2) * tau * tau * dom - d * (R(1) + e) - tau * d * de;
  dc[2] = -d + R(2) * tau * om + tau * tau * dom;
  dc[3] = om + tau * dom;
  dc[4] = d * e + tau * d * de - R(4) * tau * om - R(2) * tau * tau * dom;
  dc[5] = R(-2) * tau * om - tau * tau * dom;
}

// Vector-Jacobian product of gks_gp_flux: given cotangents gFn, gFt of (Fn, Ft), accumulates
// the cotangents of ql, dql, qr, dqr. Returns false for a non-physical state.
template <class R>
GKS_HD bool gks_gp_flux_vjp(const FluxParams<R>& P, const R ql[5], const R dql[3][5], const R qr[5],
                            const R dqr[3][5], R dt, const R gFn[5], const R gFt[5], R gql[5],
                            R gdql[3][5], R gqr[5], R gdqr[3][5]) {
  // ---------------- forward recomputation
  Prim<R> wl, wr, w0;
  bool ok = to_prim(ql, P.gamma, wl) & to_prim(qr, P.gamma, wr);
  if (!ok) return false;
  Mom<R> Mlp, Mrn;
  maxwell_moments(wl.U, wl.V, wl.W, wl.lam, P.K, +1, Mlp);
  maxwell_moments(wr.U, wr.V, wr.W, wr.lam, P.K, -1, Mrn);
  R q0[5], Gl0[5], Gr0[5];
  G(Mlp, 0, 0, 0, 0, Gl0);
  G(Mrn, 0, 0, 0, 0, Gr0);
#pragma unroll
  for (int q = 0; q < 5; ++q) q0[q] = wl.rho * Gl0[q] + wr.rho * Gr0[q];
  if (!to_prim(q0, P.gamma, w0)) return false;
  Mom<R> M0;
  maxwell_moments(w0.U, w0.V, w0.W, w0.lam, P.K, 0, M0);
  R al[3][5], ar[3][5], bl[3][5], br[3][5];
  const R irl = R(1) / wl.rho, irr = R(1) / wr.rho;
  for (int d = 0; d < 3; ++d) {
    for (int q = 0; q < 5; ++q) {
      bl[d][q] = dql[d][q] * irl;
      br[d][q] = dqr[d][q] * irr;
    }
    slope_solve(wl.U, wl.V, wl.W, wl.lam, P.K, bl[d], al[d]);
    slope_solve(wr.U, wr.V, wr.W, wr.lam, P.K, br[d], ar[d]);
  }
  R ab[3][5], bb[3][5], sl[3][5], sr[3][5], Ab[5], bA[5];
  const R ir0 = R(1) / w0.rho;
  for (int d = 0; d < 3; ++d) {
    Ga(Mlp, al[d], 0, 0, 0, sl[d]);
    Ga(Mrn, ar[d], 0, 0, 0, sr[d]);
    for (int q = 0; q < 5; ++q) bb[d][q] = (wl.rho * sl[d][q] + wr.rho * sr[d][q]) * ir0;
    slope_solve(w0.U, w0.V, w0.W, w0.lam, P.K, bb[d], ab[d]);
  }
  Gadotu(M0, ab, 0, bA);
  for (int q = 0; q < 5; ++q) bA[q] = -bA[q];
  slope_solve(w0.U, w0.V, w0.W, w0.lam, P.K, bA, Ab);
  const R xdp = (wl.p - wr.p) / (wl.p + wr.p);
  const R dp = k_abs(xdp);
  const R tau = collision_time(P, w0.p, R(1) / w0.rho, dp, dt);
  R e0[5], e1[5], e2[5];
  G(M0, 1, 0, 0, 0, e0);
  Ga(M0, Ab, 1, 0, 0, e2);
  if (P.tau_model != 0) {
    Gadotu(M0, ab, 1, e1);
  } else {
    for (int q = 0; q < 5; ++q) e1[q] = R(0);
  }
  // ---------------- reverse
  PrimAdj<R> gwl, gwr, gw0;
  Mom<R> gMlp, gMrn, gM0;
  mom_zero(gMlp);
  mom_zero(gMrn);
  mom_zero(gM0);
  R gal[3][5], gar[3][5], gab[3][5], gAb[5];
  for (int d = 0; d < 3; ++d)
    for (int q = 0; q < 5; ++q) gal[d][q] = gar[d][q] = gab[d][q] = R(0);
  for (int q = 0; q < 5; ++q) gAb[q] = R(0);
  R ge0[5], ge1[5], ge2[5], gtau = R(0);
  if (!P.full) {
    for (int q = 0; q < 5; ++q) {
      gw0.rho += gFn[q] * (e0[q] - tau * (e1[q] + e2[q])) + gFt[q] * e2[q];
      ge0[q] = w0.rho * gFn[q];
      ge1[q] = -w0.rho * tau * gFn[q];
      ge2[q] = -w0.rho * tau * gFn[q] + w0.rho * gFt[q];
      gtau += -w0.rho * gFn[q] * (e1[q] + e2[q]);
    }
  } else {
    Mom<R> Ml, Mr;
    maxwell_moments(wl.U, wl.V, wl.W, wl.lam, P.K, 0, Ml);
    maxwell_moments(wr.U, wr.V, wr.W, wr.lam, P.K, 0, Mr);
    R bAl[5], bAr[5], Al[5], Ar[5];
    Gadotu(Ml, al, 0, bAl);
    Gadotu(Mr, ar, 0, bAr);
    for (int q = 0; q < 5; ++q) {
      bAl[q] = -bAl[q];
      bAr[q] = -bAr[q];
    }
    slope_solve(wl.U, wl.V, wl.W, wl.lam, P.K, bAl, Al);
    slope_solve(wr.U, wr.V, wr.W, wr.lam, P.K, bAr, Ar);
    R cn[6], ct[6], ch[6], cf[6];
    const bool tpos = tau > R(0);
    if (tpos) {
      flux1_integrals(tau, R(0.5) * dt, ch);
      flux1_integrals(tau, dt, cf);
      for (int q = 0; q < 6; ++q) {
        cn[q] = (R(4) * ch[q] - cf[q]) / dt;
        ct[q] = R(4) * (cf[q] - R(2) * ch[q]) / (dt * dt);
      }
    } else {
      for (int q = 0; q < 6; ++q) cn[q] = ct[q] = R(0);
      cn[0] = R(1);
      ct[2] = R(1);
    }
    R nl0[5], nl1[5], nl2[5], nr0[5], nr1[5], nr2[5];
    G(Mlp, 1, 0, 0, 0, nl0);
    Gadotu(Mlp, al, 1, nl1);
    Ga(Mlp, Al, 1, 0, 0, nl2);
    G(Mrn, 1, 0, 0, 0, nr0);
    Gadotu(Mrn, ar, 1, nr1);
    Ga(Mrn, Ar, 1, 0, 0, nr2);
    // Fn = rho0 (cn0 e0 + cn1 e1 + cn2 e2) + rhol (cn3 nl0 + cn4 nl1 + cn5 nl2) + rhor (...)
    R gcn[6] = {R(0), R(0), R(0), R(0), R(0), R(0)}, gct[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
    R gnl0[5], gnl1[5], gnl2[5], gnr0[5], gnr1[5], gnr2[5];
    for (int q = 0; q < 5; ++q) {
      const R En = cn[0] * e0[q] + cn[1] * e1[q] + cn[2] * e2[q];
      const R Et = ct[0] * e0[q] + ct[1] * e1[q] + ct[2] * e2[q];
      const R Ln = cn[3] * nl0[q] + cn[4] * nl1[q] + cn[5] * nl2[q];
      const R Lt = ct[3] * nl0[q] + ct[4] * nl1[q] + ct[5] * nl2[q];
      const R Rn = cn[3] * nr0[q] + cn[4] * nr1[q] + cn[5] * nr2[q];
      const R Rt = ct[3] * nr0[q] + ct[4] * nr1[q] + ct[5] * nr2[q];
      gw0.rho += gFn[q] * En + gFt[q] * Et;
      gwl.rho += gFn[q] * Ln + gFt[q] * Lt;
      gwr.rho += gFn[q] * Rn + gFt[q] * Rt;
      ge0[q] = w0.rho * (cn[0] * gFn[q] + ct[0] * gFt[q]);
      ge1[q] = w0.rho * (cn[1] * gFn[q] + ct[1] * gFt[q]);
      ge2[q] = w0.rho * (cn[2] * gFn[q] + ct[2] * gFt[q]);
      gnl0[q] = wl.rho * (cn[3] * gFn[q] + ct[3] * gFt[q]);
      gnl1[q] = wl.rho * (cn[4] * gFn[q] + ct[4] * gFt[q]);
      gnl2[q] = wl.rho * (cn[5] * gFn[q] + ct[5] * gFt[q]);
      gnr0[q] = wr.rho * (cn[3] * gFn[q] + ct[3] * gFt[q]);
      gnr1[q] = wr.rho * (cn[4] * gFn[q] + ct[4] * gFt[q]);
      gnr2[q] = wr.rho * (cn[5] * gFn[q] + ct[5] * gFt[q]);
      gcn[0] += gFn[q] * w0.rho * e0[q];
      gcn[1] += gFn[q] * w0.rho * e1[q];
      gcn[2] += gFn[q] * w0.rho * e2[q];
      gcn[3] += gFn[q] * (wl.rho * nl0[q] + wr.rho * nr0[q]);
      gcn[4] += gFn[q] * (wl.rho * nl1[q] + wr.rho * nr1[q]);
      gcn[5] += gFn[q] * (wl.rho * nl2[q] + wr.rho * nr2[q]);
      gct[0] += gFt[q] * w0.rho * e0[q];
      gct[1] += gFt[q] * w0.rho * e1[q];
      gct[2] += gFt[q] * w0.rho * e2[q];
      gct[3] += gFt[q] * (wl.rho * nl0[q] + wr.rho * nr0[q]);
      gct[4] += gFt[q] * (wl.rho * nl1[q] + wr.rho * nr1[q]);
      gct[5] += gFt[q] * (wl.rho * nl2[q] + wr.rho * nr2[q]);
    }
    if (tpos) {
      R dch[6], dcf[6];
      flux1_integrals_dtau(tau, R(0.5) * dt, dch);
      flux1_integrals_dtau(tau, dt, dcf);
      for (int q = 0; q < 6; ++q)
        gtau += gcn[q] * (R(4) * dch[q] - dcf[q]) / dt +
                gct[q] * R(4) * (dcf[q] - R(2) * dch[q]) / (dt * dt);
    }
    // non-equilibrium moments
    G_adj(Mlp, gMlp, 1, 0, 0, 0, gnl0);
    Gadotu_adj(Mlp, al, 1, gnl1, gMlp, gal);
    R gAl[5] = {R(0), R(0), R(0), R(0), R(0)}, gAr[5] = {R(0), R(0), R(0), R(0), R(0)};
    Ga_adj(Mlp, Al, 1, 0, 0, gnl2, gMlp, gAl);
    G_adj(Mrn, gMrn, 1, 0, 0, 0, gnr0);
    Gadotu_adj(Mrn, ar, 1, gnr1, gMrn, gar);
    Ga_adj(Mrn, Ar, 1, 0, 0, gnr2, gMrn, gAr);
    // A^{l,r} = slope(w_{l,r}, -<(a.u) psi>_{l,r})
    R gbAl[5] = {R(0), R(0), R(0), R(0), R(0)}, gbAr[5] = {R(0), R(0), R(0), R(0), R(0)};
    slope_solve_adj(wl.U, wl.V, wl.W, wl.lam, P.K, bAl, gAl, gwl.U, gwl.V, gwl.W, gwl.lam, gbAl);
    slope_solve_adj(wr.U, wr.V, wr.W, wr.lam, P.K, bAr, gAr, gwr.U, gwr.V, gwr.W, gwr.lam, gbAr);
    Mom<R> gMl, gMr;
    mom_zero(gMl);
    mom_zero(gMr);
    for (int q = 0; q < 5; ++q) {
      gbAl[q] = -gbAl[q];
      gbAr[q] = -gbAr[q];
    }
    Gadotu_adj(Ml, al, 0, gbAl, gMl, gal);
    Gadotu_adj(Mr, ar, 0, gbAr, gMr, gar);
    maxwell_moments_adj(wl.U, wl.V, wl.W, wl.lam, P.K, 0, Ml, gMl, gwl.U, gwl.V, gwl.W, gwl.lam);
    maxwell_moments_adj(wr.U, wr.V, wr.W, wr.lam, P.K, 0, Mr, gMr, gwr.U, gwr.V, gwr.W, gwr.lam);
  }
  // equilibrium flux moments
  G_adj(M0, gM0, 1, 0, 0, 0, ge0);
  Ga_adj(M0, Ab, 1, 0, 0, ge2, gM0, gAb);
  if (P.tau_model != 0) Gadotu_adj(M0, ab, 1, ge1, gM0, gab);
  // collision time
  if (P.tau_model != 0) {
    R gdp = gtau * P.tau_C * dt;
    if (P.tau_model == 2) gw0.p += -gtau * P.mu / (w0.p * w0.p);
    if (P.tau_model == 3) {
      // tau_mu = mu (T0/T_ref)^s / p0, T0 = p0/rho0: d/dp0 = (s - 1) tau_mu / p0,
      // d/drho0 = -s tau_mu / rho0
      const R tmu = P.mu * k_pow(w0.p / (w0.rho * P.T_ref), P.mu_pow) / w0.p;
      gw0.p += gtau * (P.mu_pow - R(1)) * tmu / w0.p;
      gw0.rho += -gtau * P.mu_pow * tmu / w0.rho;
    }
    const R gx = xdp < R(0) ? -gdp : gdp;
    const R s = wl.p + wr.p;
    gwl.p += gx * R(2) * wr.p / (s * s);
    gwr.p += gx * R(-2) * wl.p / (s * s);
  }
  // Ab = slope(w0, -<(ab.u) psi>_0)
  {
    R gbA[5] = {R(0), R(0), R(0), R(0), R(0)};
    slope_solve_adj(w0.U, w0.V, w0.W, w0.lam, P.K, bA, gAb, gw0.U, gw0.V, gw0.W, gw0.lam, gbA);
    for (int q = 0; q < 5; ++q) gbA[q] = -gbA[q];
    Gadotu_adj(M0, ab, 0, gbA, gM0, gab);
  }
  // ab[d] = slope(w0, (rhol <al psi>_+ + rhor <ar psi>_-) / rho0)
  for (int d = 0; d < 3; ++d) {
    R gbb[5] = {R(0), R(0), R(0), R(0), R(0)};
    slope_solve_adj(w0.U, w0.V, w0.W, w0.lam, P.K, bb[d], gab[d], gw0.U, gw0.V, gw0.W, gw0.lam, gbb);
    R gsl[5], gsr[5];
    for (int q = 0; q < 5; ++q) {
      gwl.rho += gbb[q] * sl[d][q] * ir0;
      gwr.rho += gbb[q] * sr[d][q] * ir0;
      gw0.rho += -gbb[q] * bb[d][q] * ir0;
      gsl[q] = gbb[q] * wl.rho * ir0;
      gsr[q] = gbb[q] * wr.rho * ir0;
    }
    Ga_adj(Mlp, al[d], 0, 0, 0, gsl, gMlp, gal[d]);
    Ga_adj(Mrn, ar[d], 0, 0, 0, gsr, gMrn, gar[d]);
  }
  // al[d] = slope(wl, dql[d] / rhol), same on the right
  for (int d = 0; d < 3; ++d) {
    R gbl[5] = {R(0), R(0), R(0), R(0), R(0)}, gbr[5] = {R(0), R(0), R(0), R(0), R(0)};
    slope_solve_adj(wl.U, wl.V, wl.W, wl.lam, P.K, bl[d], gal[d], gwl.U, gwl.V, gwl.W, gwl.lam, gbl);
    slope_solve_adj(wr.U, wr.V, wr.W, wr.lam, P.K, br[d], gar[d], gwr.U, gwr.V, gwr.W, gwr.lam, gbr);
    for (int q = 0; q < 5; ++q) {
      gdql[d][q] += gbl[q] * irl;
      gdqr[d][q] += gbr[q] * irr;
      gwl.rho += -gbl[q] * bl[d][q] * irl;
      gwr.rho += -gbr[q] * br[d][q] * irr;
    }
  }
  // M0 = moments(w0); w0 = prim(q0)
  maxwell_moments_adj(w0.U, w0.V, w0.W, w0.lam, P.K, 0, M0, gM0, gw0.U, gw0.V, gw0.W, gw0.lam);
  R gq0[5] = {R(0), R(0), R(0), R(0), R(0)};
  to_prim_adj(q0, P.gamma, w0, gw0, gq0);
  // q0 = rhol G(Mlp) + rhor G(Mrn)
  {
    R sgl[5], sgr[5];
    for (int q = 0; q < 5; ++q) {
      gwl.rho += gq0[q] * Gl0[q];
      gwr.rho += gq0[q] * Gr0[q];
      sgl[q] = wl.rho * gq0[q];
      sgr[q] = wr.rho * gq0[q];
    }
    G_adj(Mlp, gMlp, 0, 0, 0, 0, sgl);
    G_adj(Mrn, gMrn, 0, 0, 0, 0, sgr);
  }
  maxwell_moments_adj(wl.U, wl.V, wl.W, wl.lam, P.K, +1, Mlp, gMlp, gwl.U, gwl.V, gwl.W, gwl.lam);
  maxwell_moments_adj(wr.U, wr.V, wr.W, wr.lam, P.K, -1, Mrn, gMrn, gwr.U, gwr.V, gwr.W, gwr.lam);
  to_prim_adj(ql, P.gamma, wl, gwl, gql);
  to_prim_adj(qr, P.gamma, wr, gwr, gqr);
  return true;
}

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
  // far-field planes: the ghost is farfield_state of the owner's value only (its reverse is
  // farfield_state_vjp); gks_residual_vjp does not take such meshes, so the kernel leaves it out
  if (code >= 12) return;
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
  if (!gks_gp_flux_vjp(P, ql, dql, qr, dqr, dt, gFn, gFt, gql, gdql, gqr, gdqr)) return false;
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

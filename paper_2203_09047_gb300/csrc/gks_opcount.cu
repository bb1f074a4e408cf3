// Algorithmic operation count of one face Gauss point of the flux kernel: the same templated
// device code (polynomial evaluation of both sides, frame rotation, gas-kinetic flux, back
// rotation, weighting) instantiated on the host with a scalar type that counts its arithmetic.
// Used to state the flops per unit behind the roofline fraction of the flux kernel.
#include <cmath>
#include <cstdint>

#include "gks_kinetic.cuh"

namespace gks {
namespace opc {

struct Counter {
  int64_t flops = 0;    // +, -, *, / (an FMA counts as two)
  int64_t special = 0;  // exp, erfc, sqrt, pow
};
static Counter g_count;

struct Op {
  double v = 0.0;
  Op() = default;
  Op(double x) : v(x) {}
};
inline Op bump(double r) {
  ++g_count.flops;
  return Op(r);
}
inline Op operator+(Op a, Op b) { return bump(a.v + b.v); }
inline Op operator-(Op a, Op b) { return bump(a.v - b.v); }
inline Op operator*(Op a, Op b) { return bump(a.v * b.v); }
inline Op operator/(Op a, Op b) { return bump(a.v / b.v); }
inline Op operator-(Op a) { return Op(-a.v); }
inline Op& operator+=(Op& a, Op b) { a = a + b; return a; }
inline Op& operator-=(Op& a, Op b) { a = a - b; return a; }
inline Op& operator*=(Op& a, Op b) { a = a * b; return a; }
inline bool operator<(Op a, Op b) { return a.v < b.v; }
inline bool operator>(Op a, Op b) { return a.v > b.v; }
inline bool operator!=(Op a, Op b) { return a.v != b.v; }
inline Op k_exp(Op a) { ++g_count.special; return Op(std::exp(a.v)); }
inline Op k_erfc(Op a) { ++g_count.special; return Op(std::erfc(a.v)); }
inline Op k_sqrt(Op a) { ++g_count.special; return Op(std::sqrt(a.v)); }
inline Op k_pow(Op a, Op b) { ++g_count.special; return Op(std::pow(a.v, b.v)); }
inline Op k_abs(Op a) { return Op(std::fabs(a.v)); }

struct ArrCoef {
  const Op (*c)[10];
  Op operator()(int v, int j) const { return c[v][j]; }
};

}  // namespace opc
}  // namespace gks

extern "C" int gks_flux_opcount(int flux_mode, int tau_model, double* flops, double* special) {
  using namespace gks;
  using opc::Op;
  FluxParams<Op> P;
  P.gamma = 1.4;
  P.K = 2.0;
  P.mu = 1e-3;
  P.tau_eps = 0.01;
  P.tau_C = 1.0;
  P.full = flux_mode;
  P.tau_model = tau_model;
  // a smooth, physical pair of reconstructions at an oblique face
  Op cl[5][10], cr[5][10];
  const double base[5] = {1.1, 0.3, -0.2, 0.4, 2.9};
  for (int v = 0; v < 5; ++v)
    for (int j = 0; j < 10; ++j) {
      cl[v][j] = Op(j == 0 ? base[v] : 0.01 * (j + v));
      cr[v][j] = Op(j == 0 ? base[v] * 1.01 : -0.01 * (j + 2 * v));
    }
  Op dl[3] = {Op(0.01), Op(-0.02), Op(0.015)}, dr[3] = {Op(-0.02), Op(0.01), Op(-0.005)};
  Op n1[3] = {Op(0.48), Op(0.6), Op(0.64)};
  opc::g_count = opc::Counter();
  Op vl[5], gl[5][3], vr[5], gr[5][3], acc[10];
  eval_poly(opc::ArrCoef{cl}, dl, vl, gl);
  eval_poly(opc::ArrCoef{cr}, dr, vr, gr);
  const bool ok = gp_flux_global(P, vl, gl, vr, gr, n1, Op(0.01), Op(1e-3), acc);
  // the four Gauss points of a face are summed: 10 additions per point
  *flops = (double)opc::g_count.flops + 10.0;
  *special = (double)opc::g_count.special;
  return ok ? 0 : 1;
}

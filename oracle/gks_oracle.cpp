// Oracle for the third-order gas-kinetic scheme on hybrid unstructured meshes
// (Yang, Pan & Xu, arXiv 2203.09047).
//
// TEST INFRASTRUCTURE ONLY. This is a plain, slow, FP64 CPU restatement of the method, written
// to check the CUDA library against. Only the tests, the smoke check and the CPU-baseline leg of
// the benchmark load it. It shares no code with the CUDA library: it does its own face matching,
// stencil selection, quadrature, least squares and kinetic moments, each straight from the
// definitions in the paper, with no precomputed pseudo-inverses, no closed-form slope solves and
// no fused evaluation.
//
// Readings of points the paper leaves open (the CUDA path follows the same readings):
//  * face Gauss points at (+-sqrt(3)/6, +-sqrt(3)/6) on [-1/2,1/2]^2 (Eq. flux-qud prints
//    sqrt(3)/3 for a domain of side 1);
//  * 3-point Gauss-Legendre per direction on [-1/2,1/2] for the volume integrals (Section 2);
//  * the cyclic vertex lists of cells and faces map to the tensor slots (-,-,-) (+,-,-) (+,+,-)
//    (-,+,-) (-,-,+) (+,-,+) (+,+,+) (-,+,+) of the trilinear map and (-,-) (-,+) (+,+) (+,-) of
//    the bilinear map;
//  * prism face F3 is {p1 p2 p5 p4} (the printed {p1 p2 p6 p4} is not a face of the prism);
//  * a face's vertex list is oriented so that X_eta x X_zeta points out of its owner (the lower
//    cell index), then rotated so the smallest owner-side node id comes first; a triangle
//    (a,b,c) becomes the quadrilateral (a,b,c,c);
//  * neighbours-of-neighbours of a neighbour with more than three other faces: all of them, in
//    face-label order; every stencil is a set (first occurrence kept) of (cell, transform)
//    pairs and excludes the cell itself; least squares are unweighted;
//  * WENO: epsilon and the exponent of tau/(beta+epsilon) are parameters (defaults 1e-8 and 1);
//  * Eq. flux-2 is read as g0 [1 - tau (a.u + A) + t A];
//  * time integrals F(dt/2), F(dt) of the face flux give F^n and dF/dt by the two-point fit;
//  * two-stage fourth-order update: Q* = Q + dt/2 L + dt^2/8 Lt,
//    Q^{n+1} = Q + dt L + dt^2/6 (Lt + 2 Lt*) (Section 3.3, the cited two-stage method);
//  * reflecting (slip) walls: the ghost is the mirror image of the owner; the wall flux has its
//    mass, energy and tangential-momentum components set to zero;
//  * no-slip walls (Section 5 names adiabatic and isothermal ones, without formulas): ghost cells
//    in the stencils carry all three velocity components negated (the stationary adiabatic
//    wall); at the wall's Gauss points the ghost is rho_g = rho, U_g = 2 U_w - U with p_g = p
//    (adiabatic) or T_g = 2 T_w - p/rho (isothermal), its gradient the mirrored gradient mapped
//    by the Jacobian of that map; the wall flux has no mass component and, at an adiabatic wall,
//    the energy component U_w . (momentum flux);
//  * far field (Section 5.4, Riemann invariants): the ghost, in the stencils and at the Gauss
//    points, is the characteristic boundary state of the source or owner state and the far
//    field (R+ from inside, R- from the far field, entropy and tangential velocity from the
//    upwind side; supersonic in- and outflow take one side whole), with no gradient at the
//    Gauss points; its face flux is the plain GKS flux;
//  * power-law viscosity (Section 5.4): tau = mu (T0/T_ref)^mu_pow / p0 + C dp dt with
//    T0 = p0 / rho0 of the interface equilibrium;
//  * implicit step (Section 4): the system is written with |Omega_i| (the printed Eq. jacobi
//    drops the volume of the residual's definition), Res is the GKS residual averaged over the
//    step, r_f = max over both sides of |U . n| + c at Q^n, S_f n_f the face's area vector.

#include <omp.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

namespace {

// ---------------------------------------------------------------------------------------------
// Scalars. The state-dependent part is templated so that the same code also runs on forward
// dual numbers (value + one directional derivative) for gradient checks.
struct Dual {
  double v = 0.0, d = 0.0;
  Dual() = default;
  Dual(double a) : v(a), d(0.0) {}
  Dual(double a, double b) : v(a), d(b) {}
};
inline Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
inline Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
inline Dual operator-(Dual a) { return {-a.v, -a.d}; }
inline Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
inline Dual operator/(Dual a, Dual b) { return {a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)}; }
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
inline Dual& operator*=(Dual& a, Dual b) { a = a * b; return a; }
inline Dual& operator/=(Dual& a, Dual b) { a = a / b; return a; }
inline Dual exp(Dual a) { double e = std::exp(a.v); return {e, e * a.d}; }
inline Dual sqrt(Dual a) { double s = std::sqrt(a.v); return {s, a.d / (2.0 * s)}; }
inline Dual erfc(Dual a) {
  return {std::erfc(a.v), -2.0 / std::sqrt(M_PI) * std::exp(-a.v * a.v) * a.d};
}
inline Dual fabs(Dual a) { return a.v < 0 ? -a : a; }
inline double val(double a) { return a; }
inline double val(Dual a) { return a.v; }
inline Dual pow(Dual a, double e) {
  const double p = std::pow(a.v, e);
  return {p, e * p / a.v * a.d};
}
using std::pow;
using std::exp;
using std::sqrt;
using std::erfc;
using std::fabs;

// ---------------------------------------------------------------------------------------------
// Affine per-axis transforms x' = s x + t (periodic shifts and mirror images).
// The flow variables of an image carry the boundary conditions of the wall planes it was
// reflected across (Section 2: ghost geometry by mirror images, flow variables from the boundary
// condition). `walls` lists those planes (axis + 3 side) in the order the reflections apply;
// bit j of vflip records whether the j-th velocity component ends up negated. Images that
// coincide geometrically are one member (the first path found is kept).
struct Xform {
  double s[3] = {1, 1, 1};
  double t[3] = {0, 0, 0};
  int vflip = 0;
  int nw = 0, walls[8];  // at most two walls per member: a face and a face of a neighbour
};
Xform compose(const Xform& a, const Xform& b) {  // a after b
  Xform c;
  for (int k = 0; k < 3; ++k) {
    c.s[k] = a.s[k] * b.s[k];
    c.t[k] = a.s[k] * b.t[k] + a.t[k];
  }
  c.vflip = a.vflip ^ b.vflip;
  for (int k = 0; k < b.nw && c.nw < 8; ++k) c.walls[c.nw++] = b.walls[k];
  for (int k = 0; k < a.nw && c.nw < 8; ++k) c.walls[c.nw++] = a.walls[k];
  return c;
}
bool same_xform(const Xform& a, const Xform& b, double tol) {
  for (int k = 0; k < 3; ++k)
    if (a.s[k] != b.s[k] || std::fabs(a.t[k] - b.t[k]) > tol) return false;
  return true;
}
bool is_identity(const Xform& a, double tol) { return same_xform(a, Xform(), tol); }
void apply(const Xform& a, const double* x, double* y) {
  for (int k = 0; k < 3; ++k) y[k] = a.s[k] * x[k] + a.t[k];
}

// ---------------------------------------------------------------------------------------------
// Cell and face labels, Section 2. Paper vertex p_j sits in these degenerate-hex slots.
const int kTet = 4, kPyr = 5, kPri = 6, kHex = 8;
int vertex_slot(int type, int p) {  // p is 0-based paper label
  static const int tet[4] = {0, 1, 2, 4};
  static const int pyr[5] = {0, 1, 2, 3, 4};
  static const int pri[6] = {0, 1, 2, 4, 5, 6};
  if (type == kTet) return tet[p];
  if (type == kPyr) return pyr[p];
  if (type == kPri) return pri[p];
  return p;
}
// Face lists F_1.. in paper labels (1-based), 0-terminated.
const std::vector<std::vector<int>>& face_list(int type) {
  static const std::vector<std::vector<int>> tet = {{1, 2, 3}, {1, 2, 4}, {2, 3, 4}, {3, 1, 4}};
  static const std::vector<std::vector<int>> pyr = {
      {1, 2, 5}, {2, 3, 5}, {3, 4, 5}, {4, 1, 5}, {1, 2, 3, 4}};
  static const std::vector<std::vector<int>> pri = {
      {1, 2, 3}, {4, 5, 6}, {1, 2, 5, 4}, {2, 3, 6, 5}, {3, 1, 4, 6}};
  static const std::vector<std::vector<int>> hex = {{1, 2, 3, 4}, {1, 2, 6, 5}, {2, 3, 7, 6},
                                                    {3, 4, 8, 7}, {4, 1, 5, 8}, {5, 6, 7, 8}};
  if (type == kTet) return tet;
  if (type == kPyr) return pyr;
  if (type == kPri) return pri;
  return hex;
}

// Gauss rules on [-1/2, 1/2].
const double kG3x[3] = {-0.5 * 0.7745966692414834, 0.0, 0.5 * 0.7745966692414834};
const double kG3w[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
const double kG2x[2] = {-0.28867513459481287, 0.28867513459481287};  // sqrt(3)/6

// Trilinear map of a degenerate hexahedron, Eq. trilinear, slot order above.
const int kSlotSign[8][3] = {{-1, -1, -1}, {1, -1, -1}, {1, 1, -1}, {-1, 1, -1},
                             {-1, -1, 1},  {1, -1, 1},  {1, 1, 1},  {-1, 1, 1}};
void trilinear(const double X[8][3], double xi, double eta, double zeta, double x[3],
               double J[3][3]) {
  const double q[3] = {xi, eta, zeta};
  for (int a = 0; a < 3; ++a) {
    x[a] = 0;
    for (int b = 0; b < 3; ++b) J[a][b] = 0;
  }
  for (int s = 0; s < 8; ++s) {
    double f[3], df[3];
    for (int d = 0; d < 3; ++d) {
      f[d] = 0.5 * (1.0 + 2.0 * kSlotSign[s][d] * q[d]);
      df[d] = kSlotSign[s][d];
    }
    const double psi = f[0] * f[1] * f[2];
    const double dpsi[3] = {df[0] * f[1] * f[2], f[0] * df[1] * f[2], f[0] * f[1] * df[2]};
    for (int a = 0; a < 3; ++a) {
      x[a] += X[s][a] * psi;
      for (int b = 0; b < 3; ++b) J[a][b] += X[s][a] * dpsi[b];
    }
  }
}
double det3(const double J[3][3]) {
  return J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
         J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
         J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
}

// The 27 quadrature points and weights (weight includes |J|) of a degenerate hexahedron.
struct Quad27 {
  double x[27][3];
  double w[27];
  double min_detj;
};
Quad27 quad27(const double X[8][3]) {
  Quad27 q;
  q.min_detj = 1e300;
  int n = 0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k) {
        double J[3][3];
        trilinear(X, kG3x[i], kG3x[j], kG3x[k], q.x[n], J);
        const double dj = det3(J);
        q.min_detj = std::min(q.min_detj, dj);
        q.w[n] = kG3w[i] * kG3w[j] * kG3w[k] * dj;
        ++n;
      }
  return q;
}

// The nine monomials x^n, |n| = 1..2, in the order (x, y, z, xx, yy, zz, xy, xz, yz).
const int kMono[9][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {2, 0, 0}, {0, 2, 0},
                         {0, 0, 2}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}};
double ipow(double x, int n) { return n == 0 ? 1.0 : n == 1 ? x : x * x; }
double monomial(int n, const double* y) {
  return ipow(y[0], kMono[n][0]) * ipow(y[1], kMono[n][1]) * ipow(y[2], kMono[n][2]);
}
// d/dy_a of monomial n
double dmonomial(int n, int a, const double* y) {
  int e[3] = {kMono[n][0], kMono[n][1], kMono[n][2]};
  if (e[a] == 0) return 0.0;
  const double c = e[a];
  e[a] -= 1;
  return c * ipow(y[0], e[0]) * ipow(y[1], e[1]) * ipow(y[2], e[2]);
}
// d2/dy_a dy_b of monomial n
double d2monomial(int n, int a, int b, const double* y) {
  int e[3] = {kMono[n][0], kMono[n][1], kMono[n][2]};
  double c = 1.0;
  if (e[a] == 0) return 0.0;
  c *= e[a];
  e[a] -= 1;
  if (e[b] == 0) return 0.0;
  c *= e[b];
  e[b] -= 1;
  return c * ipow(y[0], e[0]) * ipow(y[1], e[1]) * ipow(y[2], e[2]);
}

// ---------------------------------------------------------------------------------------------
// Least squares by Householder QR (column-major m x n, m >= n). Returns false if rank < n.
struct QR {
  int m = 0, n = 0;
  std::vector<double> a;     // Householder vectors below the diagonal, R on/above
  std::vector<double> beta;  // reflector scalars
  std::vector<double> rdiag;
};
bool qr_factor(const std::vector<double>& A, int m, int n, QR& qr) {
  qr.m = m;
  qr.n = n;
  qr.a = A;
  qr.beta.assign(n, 0.0);
  qr.rdiag.assign(n, 0.0);
  double scale = 0.0;
  for (double v : A) scale = std::max(scale, std::fabs(v));
  if (m < n) return false;
  for (int k = 0; k < n; ++k) {
    double nrm = 0.0;
    for (int i = k; i < m; ++i) nrm += qr.a[i + k * m] * qr.a[i + k * m];
    nrm = std::sqrt(nrm);
    if (nrm <= 1e-12 * std::max(scale, 1e-300)) return false;
    const double alpha = qr.a[k + k * m] > 0 ? -nrm : nrm;
    qr.a[k + k * m] -= alpha;  // v = x - alpha e1
    double vtv = 0.0;
    for (int i = k; i < m; ++i) vtv += qr.a[i + k * m] * qr.a[i + k * m];
    qr.beta[k] = vtv > 0 ? 2.0 / vtv : 0.0;
    for (int j = k + 1; j < n; ++j) {
      double s = 0.0;
      for (int i = k; i < m; ++i) s += qr.a[i + k * m] * qr.a[i + j * m];
      s *= qr.beta[k];
      for (int i = k; i < m; ++i) qr.a[i + j * m] -= s * qr.a[i + k * m];
    }
    qr.rdiag[k] = alpha;
  }
  return true;
}
// Least-squares solution x (n) of A x ~ b (m).
template <class T>
void qr_solve(const QR& qr, const T* b, T* x) {
  const int m = qr.m, n = qr.n;
  std::vector<T> y(b, b + m);
  for (int k = 0; k < n; ++k) {
    T s = T(0.0);
    for (int i = k; i < m; ++i) s += qr.a[i + k * m] * y[i];
    s = s * qr.beta[k];
    for (int i = k; i < m; ++i) y[i] -= s * qr.a[i + k * m];
  }
  for (int k = n - 1; k >= 0; --k) {
    T s = y[k];
    for (int j = k + 1; j < n; ++j) s -= qr.a[k + j * m] * x[j];
    x[k] = s / qr.rdiag[k];
  }
}

// Dense 5x5 linear solve by Gaussian elimination with partial pivoting.
template <class T>
void solve5(T A[5][5], T b[5], T x[5]) {
  int piv[5] = {0, 1, 2, 3, 4};
  for (int k = 0; k < 5; ++k) {
    int p = k;
    for (int i = k + 1; i < 5; ++i)
      if (std::fabs(val(A[piv[i]][k])) > std::fabs(val(A[piv[p]][k]))) p = i;
    std::swap(piv[k], piv[p]);
    for (int i = k + 1; i < 5; ++i) {
      const T f = A[piv[i]][k] / A[piv[k]][k];
      for (int j = k; j < 5; ++j) A[piv[i]][j] -= f * A[piv[k]][j];
      b[piv[i]] -= f * b[piv[k]];
    }
  }
  for (int k = 4; k >= 0; --k) {
    T s = b[piv[k]];
    for (int j = k + 1; j < 5; ++j) s -= A[piv[k]][j] * x[j];
    x[k] = s / A[piv[k]][k];
  }
}

// ---------------------------------------------------------------------------------------------
// Parameters (flat array from the caller).
struct Params {
  double gamma, mu, Pr;
  int flux_mode;  // 0 smooth (Eq. flux-2), 1 full (Eq. flux-1)
  int tau_model;  // 0 zero, 1 inviscid, 2 viscous, 3 viscous with power-law mu(T)
  double tau_eps, tau_C;
  double weno_gamma, weno_eps;
  int weno_pow;
  int weno_linear;  // 1: use the linear weights (omega-bar = gamma), i.e. plain P0
  double T_ref, mu_pow;   // mu(T) = mu (T / T_ref)^mu_pow, T = p / rho (Section 5.4)
  double uw[6][3], Tw[6];  // per wall plane (axis + 3 side): velocity, temperature (<= 0: adiabatic)
  double finf[6][5];       // far-field state per plane: rho, U, V, W, p
  int gp_fallback;  // 1: a side whose reconstructed state at a Gauss point has rho <= 0 or
                    // p <= 0 takes its cell average with zero gradient (not in the paper)
};
Params read_params(const double* p) {
  Params q;
  q.gamma = p[0];
  q.mu = p[1];
  q.Pr = p[2];
  q.flux_mode = (int)p[3];
  q.tau_model = (int)p[4];
  q.tau_eps = p[5];
  q.tau_C = p[6];
  q.weno_gamma = p[7];
  q.weno_eps = p[8];
  q.weno_pow = (int)p[9];
  q.weno_linear = (int)p[10];
  q.T_ref = p[11];
  q.mu_pow = p[12];
  for (int w = 0; w < 6; ++w) {
    for (int a = 0; a < 3; ++a) q.uw[w][a] = p[13 + 4 * w + a];
    q.Tw[w] = p[13 + 4 * w + 3];
  }
  for (int w = 0; w < 6; ++w)
    for (int v = 0; v < 5; ++v) q.finf[w][v] = p[37 + 5 * w + v];
  q.gp_fallback = (int)p[67];
  return q;
}

// ---------------------------------------------------------------------------------------------
// Mesh: topology, geometry, stencils (Section 2 and Section 3.1).
struct Member {
  int cell;
  Xform T;  // maps the member cell's own coordinates into the target cell's frame
};
struct Face {
  int owner = -1, owner_face = -1, nb = -1, nb_face = -1;
  Xform nb_to_owner;  // neighbour frame -> owner frame (for a wall: the mirror image)
  int wall_axis = -1;
  int wall_kind = 0;   // 1 slip, 2 no-slip, 3 far field (the box condition of its axis)
  int wall_plane = -1;  // axis + 3 side (side 1: the upper plane)
  double xg[4][3], n[4][3], w[4];  // Gauss points (owner frame), unit normals, area weights
  double area = 0.0;
};
struct Cell {
  int type = 0;
  int node[8];
  double X[8][3];
  std::vector<int> face_id;
  std::vector<Member> nbs;  // neighbour across each local face, in the cell's frame
  double vol = 0, centroid[3], h = 0;
  double mean_mono[9];
  std::vector<Member> stencil;            // S_i without the cell itself
  std::vector<std::vector<int>> sub;      // sub-stencils as indices into `stencil`
  QR qr0;
  std::vector<QR> qrm;
  bool plain = true;                      // no member carries a transform
  bool ready = false;                     // stencil and least-squares systems built
};
struct Mesh {
  int n_nodes = 0, n_cells = 0;
  std::vector<double> xyz;
  int bc[3];
  double lo[3], hi[3], L[3];
  std::vector<Cell> cells;
  std::vector<Face> faces;
  std::string err;
  int min_stencil = 0;  // big stencils smaller than this take a third ring (0: as printed)
};

const int ST_OK = 0, ST_INVAL = 1, ST_MESH = 4, ST_SINGULAR = 5, ST_NONPHYS = 6;

void member_vertices(const Mesh& m, const Member& mb, double Y[8][3]) {
  for (int s = 0; s < 8; ++s) apply(mb.T, m.cells[mb.cell].X[s], Y[s]);
}

// Mean over a (transformed) member cell of the scaled monomials about the target cell.
void member_means(const Mesh& m, const Cell& t, const Member& mb, double out[9]) {
  double Y[8][3];
  member_vertices(m, mb, Y);
  const Quad27 q = quad27(Y);
  double vol = 0.0;
  for (int n = 0; n < 9; ++n) out[n] = 0.0;
  for (int g = 0; g < 27; ++g) {
    double y[3];
    for (int a = 0; a < 3; ++a) y[a] = (q.x[g][a] - t.centroid[a]) / t.h;
    vol += q.w[g];
    for (int n = 0; n < 9; ++n) out[n] += q.w[g] * monomial(n, y);
  }
  for (int n = 0; n < 9; ++n) out[n] /= vol;
}

// Bilinear face map on [-1/2,1/2]^2 with the cyclic list v1..v4 in slots (-,-) (-,+) (+,+) (+,-).
void bilinear(const double V[4][3], double eta, double zeta, double x[3], double xe[3],
              double xz[3]) {
  const double se[4] = {-1, -1, 1, 1}, sz[4] = {-1, 1, 1, -1};
  for (int a = 0; a < 3; ++a) x[a] = xe[a] = xz[a] = 0.0;
  for (int k = 0; k < 4; ++k) {
    const double fe = 0.5 * (1 + 2 * se[k] * eta), fz = 0.5 * (1 + 2 * sz[k] * zeta);
    for (int a = 0; a < 3; ++a) {
      x[a] += V[k][a] * fe * fz;
      xe[a] += V[k][a] * se[k] * fz;
      xz[a] += V[k][a] * fe * sz[k];
    }
  }
}
void cross(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

// Sub-stencil definitions (Section 2): three face neighbours (1-based local faces) and, for
// tetrahedra and pyramids, the neighbour whose own neighbours enlarge the set.
struct SubDef {
  int f[3];
  int nn;  // 0: none
};
const std::vector<SubDef>& sub_defs(int type) {
  static const std::vector<SubDef> hex = {{{1, 2, 3}, 0}, {{1, 3, 4}, 0}, {{1, 4, 5}, 0},
                                          {{1, 5, 2}, 0}, {{6, 2, 3}, 0}, {{6, 3, 4}, 0},
                                          {{6, 4, 5}, 0}, {{6, 5, 2}, 0}};
  static const std::vector<SubDef> pri = {{{1, 3, 4}, 0}, {{1, 4, 5}, 0}, {{1, 5, 3}, 0},
                                          {{2, 3, 4}, 0}, {{2, 4, 5}, 0}, {{2, 5, 3}, 0}};
  static const std::vector<SubDef> tet = {
      {{1, 2, 3}, 1}, {{1, 2, 4}, 2}, {{2, 3, 4}, 3}, {{3, 1, 4}, 4}};
  static const std::vector<SubDef> pyr = {{{1, 2, 3}, 1}, {{2, 3, 4}, 2}, {{3, 4, 1}, 3},
                                          {{4, 1, 2}, 4}, {{1, 2, 5}, 1}, {{2, 3, 5}, 2},
                                          {{3, 4, 5}, 3}, {{4, 1, 5}, 4}};
  if (type == kHex) return hex;
  if (type == kPri) return pri;
  if (type == kTet) return tet;
  return pyr;
}

int build_cell_stencil(Mesh& m, int i);

// Topology and geometry of all cells and faces; with lazy = false also every cell's stencils.
int build_mesh(Mesh& m, bool lazy) {
  const double ext = std::max({m.L[0], m.L[1], m.L[2]});
  const double tol = 1e-9 * ext;
  // cells and their own quadrature
  for (int c = 0; c < m.n_cells; ++c) {
    Cell& cl = m.cells[c];
    if (cl.type != kTet && cl.type != kPyr && cl.type != kPri && cl.type != kHex) {
      m.err = "cell " + std::to_string(c) + ": unknown type";
      return ST_INVAL;
    }
    for (int s = 0; s < 8; ++s) {
      if (cl.node[s] < 0 || cl.node[s] >= m.n_nodes) {
        m.err = "cell " + std::to_string(c) + ": node index out of range";
        return ST_INVAL;
      }
      for (int a = 0; a < 3; ++a) cl.X[s][a] = m.xyz[3 * cl.node[s] + a];
    }
    const Quad27 q = quad27(cl.X);
    if (!(q.min_detj > 0.0)) {
      m.err = "cell " + std::to_string(c) + ": inverted or degenerate";
      return ST_MESH;
    }
    double v = 0, mx[3] = {0, 0, 0};
    for (int g = 0; g < 27; ++g) {
      v += q.w[g];
      for (int a = 0; a < 3; ++a) mx[a] += q.w[g] * q.x[g][a];
    }
    cl.vol = v;
    for (int a = 0; a < 3; ++a) cl.centroid[a] = mx[a] / v;
    cl.h = std::cbrt(v);
    for (int n = 0; n < 9; ++n) cl.mean_mono[n] = 0.0;
    for (int g = 0; g < 27; ++g) {
      double y[3];
      for (int a = 0; a < 3; ++a) y[a] = (q.x[g][a] - cl.centroid[a]) / cl.h;
      for (int n = 0; n < 9; ++n) cl.mean_mono[n] += q.w[g] * monomial(n, y) / v;
    }
  }
  // periodic images of nodes share one canonical id
  std::vector<int> canon(m.n_nodes);
  {
    std::map<std::array<long long, 3>, int> seen;
    for (int i = 0; i < m.n_nodes; ++i) {
      std::array<long long, 3> k;
      for (int a = 0; a < 3; ++a) {
        double p = m.xyz[3 * i + a];
        if (m.bc[a] == 0 && std::fabs(p - m.hi[a]) < tol) p -= m.L[a];
        k[a] = std::llround((p - m.lo[a]) / (1e-7 * ext));
      }
      auto it = seen.find(k);
      if (it == seen.end()) {
        seen.emplace(k, i);
        canon[i] = i;
      } else {
        canon[i] = it->second;
      }
    }
  }
  // faces: match local faces by their sets of canonical vertex ids
  std::map<std::vector<int>, std::vector<std::pair<int, int>>> match;
  for (int c = 0; c < m.n_cells; ++c) {
    Cell& cl = m.cells[c];
    const auto& fl = face_list(cl.type);
    cl.face_id.assign(fl.size(), -1);
    cl.nbs.assign(fl.size(), Member{-1, Xform()});
    for (int p = 0; p < (int)fl.size(); ++p) {
      std::vector<int> key;
      for (int lab : fl[p]) key.push_back(canon[cl.node[vertex_slot(cl.type, lab - 1)]]);
      std::sort(key.begin(), key.end());
      match[key].push_back({c, p});
    }
  }
  for (auto& kv : match) {
    auto inc = kv.second;
    if (inc.size() > 2) {
      m.err = "face shared by more than two cells";
      return ST_MESH;
    }
    std::sort(inc.begin(), inc.end());
    Face f;
    f.owner = inc[0].first;
    f.owner_face = inc[0].second;
    Cell& co = m.cells[f.owner];
    const auto& lab_o = face_list(co.type)[f.owner_face];
    std::vector<int> vo;
    for (int lab : lab_o) vo.push_back(co.node[vertex_slot(co.type, lab - 1)]);
    if (inc.size() == 2) {
      f.nb = inc[1].first;
      f.nb_face = inc[1].second;
      Cell& cn = m.cells[f.nb];
      const auto& lab_n = face_list(cn.type)[f.nb_face];
      double shift[3] = {0, 0, 0};
      bool first = true;
      for (int v : vo) {
        int match_node = -1;
        for (int lab : lab_n) {
          const int w = cn.node[vertex_slot(cn.type, lab - 1)];
          if (canon[w] == canon[v]) match_node = w;
        }
        double s[3];
        for (int a = 0; a < 3; ++a) s[a] = m.xyz[3 * v + a] - m.xyz[3 * match_node + a];
        if (first) {
          for (int a = 0; a < 3; ++a) shift[a] = s[a];
          first = false;
        } else {
          for (int a = 0; a < 3; ++a)
            if (std::fabs(s[a] - shift[a]) > 1e-6 * ext) {
              m.err = "periodic face vertices do not match by one translation";
              return ST_MESH;
            }
        }
      }
      for (int a = 0; a < 3; ++a) f.nb_to_owner.t[a] = std::fabs(shift[a]) < tol ? 0.0 : shift[a];
    } else {
      // a boundary face must lie on a reflecting plane of the box
      int axis = -1;
      double plane = 0;
      for (int a = 0; a < 3 && axis < 0; ++a) {
        if (m.bc[a] != 1 && m.bc[a] != 2 && m.bc[a] != 3) continue;
        for (double pl : {m.lo[a], m.hi[a]}) {
          bool on = true;
          for (int v : vo)
            if (std::fabs(m.xyz[3 * v + a] - pl) > tol) on = false;
          if (on) {
            axis = a;
            plane = pl;
            break;
          }
        }
      }
      if (axis < 0) {
        m.err = "unmatched face not on a reflecting boundary";
        return ST_MESH;
      }
      f.nb = -1;
      f.wall_axis = axis;
      f.wall_kind = m.bc[axis];
      f.wall_plane = axis + (std::fabs(plane - m.hi[axis]) <= tol ? 3 : 0);
      f.nb_to_owner.s[axis] = -1.0;
      f.nb_to_owner.t[axis] = 2.0 * plane;
      f.nb_to_owner.vflip = f.wall_kind == 1 ? 1 << axis : f.wall_kind == 2 ? 7 : 0;
      f.nb_to_owner.nw = 1;
      f.nb_to_owner.walls[0] = f.wall_plane;
    }
    // orient the owner-side vertex list outward, rotate the smallest node id first
    auto coords = [&](const std::vector<int>& ids, double V[4][3]) {
      for (int k = 0; k < 4; ++k) {
        const int id = ids[std::min<int>(k, (int)ids.size() - 1)];
        for (int a = 0; a < 3; ++a) V[k][a] = m.xyz[3 * id + a];
      }
    };
    {
      double V[4][3], x[3], xe[3], xz[3], nrm[3];
      coords(vo, V);
      bilinear(V, 0, 0, x, xe, xz);
      cross(xe, xz, nrm);
      double d = 0;
      for (int a = 0; a < 3; ++a) d += nrm[a] * (x[a] - co.centroid[a]);
      if (d < 0) std::reverse(vo.begin(), vo.end());
      const auto it = std::min_element(vo.begin(), vo.end());
      std::rotate(vo.begin(), it, vo.end());
    }
    {
      double V[4][3];
      coords(vo, V);  // a triangle repeats its last vertex
      int k = 0;
      f.area = 0;
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
          double xe[3], xz[3], nrm[3];
          bilinear(V, kG2x[i], kG2x[j], f.xg[k], xe, xz);
          cross(xe, xz, nrm);
          const double len = std::sqrt(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
          for (int a = 0; a < 3; ++a) f.n[k][a] = nrm[a] / len;
          f.w[k] = 0.25 * len;
          f.area += f.w[k];
          ++k;
        }
    }
    const int fid = (int)m.faces.size();
    co.face_id[f.owner_face] = fid;
    if (f.nb >= 0) {
      co.nbs[f.owner_face] = Member{f.nb, f.nb_to_owner};
      Xform inv;
      for (int a = 0; a < 3; ++a) {
        inv.s[a] = 1.0;
        inv.t[a] = -f.nb_to_owner.t[a];
      }
      m.cells[f.nb].face_id[f.nb_face] = fid;
      m.cells[f.nb].nbs[f.nb_face] = Member{f.owner, inv};
    } else {
      co.nbs[f.owner_face] = Member{f.owner, f.nb_to_owner};
    }
    m.faces.push_back(f);
  }
  if (lazy) return ST_OK;
  for (int i = 0; i < m.n_cells; ++i) {
    const int st = build_cell_stencil(m, i);
    if (st) return st;
  }
  return ST_OK;
}

// Stencils of cell i (Section 2): neighbours, then neighbours of neighbours, as a set; the
// sub-stencils; and the least-squares systems of both.
int build_cell_stencil(Mesh& m, int i) {
  const double tol = 1e-9 * std::max({m.L[0], m.L[1], m.L[2]});
  {
    Cell& ci = m.cells[i];
    if (ci.ready) return ST_OK;
    auto add = [&](std::vector<Member>& list, const Member& mb) -> int {
      if (mb.cell == i && is_identity(mb.T, tol)) return -1;
      for (size_t k = 0; k < list.size(); ++k)
        if (list[k].cell == mb.cell && same_xform(list[k].T, mb.T, tol)) return (int)k;
      list.push_back(mb);
      return (int)list.size() - 1;
    };
    auto second_ring = [&](int p) {  // neighbours of the neighbour across local face p
      std::vector<Member> out;
      const Member& nb = ci.nbs[p];
      const Cell& cj = m.cells[nb.cell];
      for (size_t q = 0; q < cj.nbs.size(); ++q)
        out.push_back(Member{cj.nbs[q].cell, compose(nb.T, cj.nbs[q].T)});
      return out;
    };
    ci.stencil.clear();
    for (size_t p = 0; p < ci.nbs.size(); ++p) add(ci.stencil, ci.nbs[p]);
    for (size_t p = 0; p < ci.nbs.size(); ++p)
      for (const Member& mb : second_ring((int)p)) add(ci.stencil, mb);
    // Reading (not in the paper): a big stencil with fewer than min_stencil members takes the
    // face neighbours of its members, member by member in stencil order and face by face in
    // face-label order, until it has min_stencil members, skipping images that cross more than
    // two wall planes.
    if ((int)ci.stencil.size() < m.min_stencil) {
      const size_t n2 = ci.stencil.size();
      for (size_t k = 0; k < n2 && (int)ci.stencil.size() < m.min_stencil; ++k) {
        const Member mk = ci.stencil[k];
        const Cell& cj = m.cells[mk.cell];
        for (size_t q = 0; q < cj.nbs.size() && (int)ci.stencil.size() < m.min_stencil; ++q) {
          const Xform T = compose(mk.T, cj.nbs[q].T);
          if (T.nw > 2) continue;
          add(ci.stencil, Member{cj.nbs[q].cell, T});
        }
      }
    }
    ci.plain = true;
    for (const Member& mb : ci.stencil)
      if (!is_identity(mb.T, tol)) ci.plain = false;
    ci.sub.clear();
    for (const SubDef& sd : sub_defs(ci.type)) {
      std::vector<Member> set;
      for (int k = 0; k < 3; ++k) add(set, ci.nbs[sd.f[k] - 1]);
      if (sd.nn) {
        for (const Member& mb : second_ring(sd.nn - 1)) add(set, mb);
      }
      std::vector<int> idx;
      for (const Member& mb : set) idx.push_back(add(ci.stencil, mb));
      ci.sub.push_back(idx);
    }
    // least-squares systems in the scaled, centred coordinates of the cell
    const int K = (int)ci.stencil.size();
    std::vector<double> rows(9 * (size_t)K);
    for (int k = 0; k < K; ++k) {
      double mm[9];
      member_means(m, ci, ci.stencil[k], mm);
      for (int n = 0; n < 9; ++n) rows[k + (size_t)n * K] = mm[n] - ci.mean_mono[n];
    }
    if (!qr_factor(rows, K, 9, ci.qr0)) {
      m.err = "cell " + std::to_string(i) + ": big stencil is rank deficient";
      return ST_SINGULAR;
    }
    ci.qrm.assign(ci.sub.size(), QR());
    for (size_t s = 0; s < ci.sub.size(); ++s) {
      const int ks = (int)ci.sub[s].size();
      std::vector<double> r(3 * (size_t)ks);
      for (int k = 0; k < ks; ++k)
        for (int n = 0; n < 3; ++n) r[k + (size_t)n * ks] = rows[ci.sub[s][k] + (size_t)n * K];
      if (!qr_factor(r, ks, 3, ci.qrm[s])) {
        m.err = "cell " + std::to_string(i) + ": sub-stencil " + std::to_string(s + 1) +
                " is rank deficient";
        return ST_SINGULAR;
      }
    }
    ci.ready = true;
  }
  return ST_OK;
}

// ---------------------------------------------------------------------------------------------
// WENO reconstruction (Section 2, Eqs. weno and indicator).
template <class T>
struct Recon {
  T Q0[5];
  T a[5][9];                      // P0 coefficients per variable
  std::vector<std::array<T, 3>> b[5];  // P_m coefficients per variable
  T wbar[5][17];                  // normalised weights omega-bar_0..M
  T beta[5][17];                  // smoothness indicators beta_0..M (Eq. indicator)
  T tau[5];                       // tau of the nonlinear weights
  double g0;                      // gamma_0
  double gm;                      // gamma_m
  int M;
};

// Flow variables of an image: the wall maps of its planes applied in order. Slip: the normal
// momentum negated. No-slip with velocity U_w (the reconstruction takes every no-slip wall as
// adiabatic): rho_g = rho, m_g = 2 U_w rho - m, E_g = E + 2 |U_w|^2 rho - 2 U_w . m (the same
// density and pressure, U_g = 2 U_w - U). Periodic images keep the state.
template <class T>
void transform_state(const Mesh& m, const Params& P, const Xform& X, const T* q, T* out) {
  for (int v = 0; v < 5; ++v) out[v] = q[v];
  for (int k = 0; k < X.nw; ++k) {
    const int pl = X.walls[k], ax = pl % 3;
    if (m.bc[ax] == 1) {
      out[1 + ax] = -out[1 + ax];
      continue;
    }
    if (m.bc[ax] == 3) {  // far field: the characteristic boundary state of the image's source
      double n[3] = {0, 0, 0};
      n[ax] = pl >= 3 ? 1.0 : -1.0;
      T in[5];
      for (int v = 0; v < 5; ++v) in[v] = out[v];
      farfield_state(P, pl, in, n, out);
      continue;
    }
    const double* uw = P.uw[pl];
    const double uw2 = uw[0] * uw[0] + uw[1] * uw[1] + uw[2] * uw[2];
    T um = T(0.0);
    for (int a = 0; a < 3; ++a) um += uw[a] * out[1 + a];
    out[4] = out[4] + 2.0 * uw2 * out[0] - 2.0 * um;
    for (int a = 0; a < 3; ++a) out[1 + a] = 2.0 * uw[a] * out[0] - out[1 + a];
  }
}

// Nonlinear weights of Section 2 from the indicators beta[0..M] of P0 and the M linear
// candidates: tau = sum_m |beta_0 - beta_m| / M, omega_m = gamma_m (1 + (tau / (beta_m + eps))^q)
// with gamma_m = weno_gamma for m >= 1, gamma_0 = 1 - M weno_gamma and q = weno_pow (printed: 1),
// then wbar_m = omega_m / sum_k omega_k. Returns tau.
template <class T>
T nonlinear_weights(const Params& P, int M, const T* beta, T* wbar) {
  T tau = T(0.0);
  for (int s = 1; s <= M; ++s) tau += fabs(beta[0] - beta[s]) / double(M);
  T sum = T(0.0);
  for (int s = 0; s <= M; ++s) {
    const double gam = s == 0 ? 1.0 - P.weno_gamma * M : P.weno_gamma;
    const T ratio = tau / (beta[s] + P.weno_eps);
    T pw = ratio;
    for (int e = 1; e < P.weno_pow; ++e) pw = pw * ratio;
    wbar[s] = gam * (1.0 + pw);
    sum += wbar[s];
  }
  for (int s = 0; s <= M; ++s) wbar[s] = wbar[s] / sum;
  return tau;
}

template <class T>
void reconstruct_cell(const Mesh& m, const Params& P, const T* Q, int n, int i, Recon<T>& r) {
  const Cell& ci = m.cells[i];
  const int K = (int)ci.stencil.size();
  const int M = (int)ci.sub.size();
  r.M = M;
  r.gm = P.weno_gamma;
  r.g0 = 1.0 - P.weno_gamma * M;
  for (int v = 0; v < 5; ++v) r.Q0[v] = Q[v * (size_t)n + i];
  // Q_k - Q_0 over the stencil, members brought into the cell's frame
  std::vector<T> dq(5 * (size_t)K);
  for (int k = 0; k < K; ++k) {
    const Member& mb = ci.stencil[k];
    T qk[5], qt[5];
    for (int v = 0; v < 5; ++v) qk[v] = Q[v * (size_t)n + mb.cell];
    transform_state(m, P, mb.T, qk, qt);
    for (int v = 0; v < 5; ++v) dq[k + (size_t)v * K] = qt[v] - r.Q0[v];
  }
  // cell quadrature for the smoothness indicators
  const Quad27 q = quad27(ci.X);
  const double vol = ci.vol, h = ci.h;
  for (int v = 0; v < 5; ++v) {
    qr_solve(ci.qr0, &dq[(size_t)v * K], r.a[v]);
    r.b[v].assign(M, {});
    for (int s = 0; s < M; ++s) {
      const int ks = (int)ci.sub[s].size();
      std::vector<T> rhs(ks);
      for (int k = 0; k < ks; ++k) rhs[k] = dq[ci.sub[s][k] + (size_t)v * K];
      qr_solve(ci.qrm[s], rhs.data(), r.b[v][s].data());
    }
    // beta_0: |l| = 1 and |l| = 2 derivatives of P0; beta_m: |l| = 1 of P_m
    T beta0 = T(0.0);
    std::vector<T> betam(M, T(0.0));
    for (int g = 0; g < 27; ++g) {
      double y[3];
      for (int a = 0; a < 3; ++a) y[a] = (q.x[g][a] - ci.centroid[a]) / h;
      for (int a = 0; a < 3; ++a) {
        T d = T(0.0);
        for (int nn = 0; nn < 9; ++nn) d += r.a[v][nn] * (dmonomial(nn, a, y) / h);
        beta0 += std::pow(vol, -1.0 / 3.0) * q.w[g] * d * d;
      }
      const int l2[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
      for (int l = 0; l < 6; ++l) {
        T d = T(0.0);
        for (int nn = 0; nn < 9; ++nn)
          d += r.a[v][nn] * (d2monomial(nn, l2[l][0], l2[l][1], y) / (h * h));
        beta0 += std::pow(vol, 1.0 / 3.0) * q.w[g] * d * d;
      }
      for (int s = 0; s < M; ++s)
        for (int a = 0; a < 3; ++a) {
          const T d = r.b[v][s][a] / h;
          betam[s] += std::pow(vol, -1.0 / 3.0) * q.w[g] * d * d;
        }
    }
    r.beta[v][0] = beta0;
    for (int s = 0; s < M; ++s) r.beta[v][s + 1] = betam[s];
    r.tau[v] = nonlinear_weights(P, M, r.beta[v], r.wbar[v]);
    if (P.weno_linear)
      for (int s = 0; s <= M; ++s) r.wbar[v][s] = T(s == 0 ? r.g0 : r.gm);
  }
}

// Value and gradient (physical coordinates, the cell's frame) of the combined reconstruction.
template <class T>
void eval_recon(const Mesh& m, int i, const Recon<T>& r, const double* x, T val_out[5],
                T grad_out[5][3]) {
  const Cell& ci = m.cells[i];
  double y[3];
  for (int a = 0; a < 3; ++a) y[a] = (x[a] - ci.centroid[a]) / ci.h;
  for (int v = 0; v < 5; ++v) {
    T p0 = r.Q0[v], g0[3] = {T(0.0), T(0.0), T(0.0)};
    for (int nn = 0; nn < 9; ++nn) {
      p0 += r.a[v][nn] * (monomial(nn, y) - ci.mean_mono[nn]);
      for (int a = 0; a < 3; ++a) g0[a] += r.a[v][nn] * (dmonomial(nn, a, y) / ci.h);
    }
    T val = r.wbar[v][0] * (p0 / r.g0), grd[3];
    for (int a = 0; a < 3; ++a) grd[a] = r.wbar[v][0] * (g0[a] / r.g0);
    for (int s = 0; s < r.M; ++s) {
      T pm = r.Q0[v];
      for (int a = 0; a < 3; ++a) pm += r.b[v][s][a] * (y[a] - ci.mean_mono[a]);
      val += (r.wbar[v][s + 1] - r.wbar[v][0] * (r.gm / r.g0)) * pm;
      for (int a = 0; a < 3; ++a)
        grd[a] += (r.wbar[v][s + 1] - r.wbar[v][0] * (r.gm / r.g0)) * (r.b[v][s][a] / ci.h);
    }
    val_out[v] = val;
    for (int a = 0; a < 3; ++a) grad_out[v][a] = grd[a];
  }
}

// ---------------------------------------------------------------------------------------------
// Gas-kinetic flux at one Gauss point (Section 3.2, Eqs. flux-1 / flux-2), in the local frame
// (u along n1). Moments are taken term by term from polynomials in (u, v, w, xi^2).
template <class T>
struct Poly {
  std::vector<std::pair<std::array<int, 4>, T>> t;
};
template <class T>
Poly<T> psi(int i) {
  Poly<T> p;
  if (i == 0) p.t.push_back({{0, 0, 0, 0}, T(1.0)});
  if (i == 1) p.t.push_back({{1, 0, 0, 0}, T(1.0)});
  if (i == 2) p.t.push_back({{0, 1, 0, 0}, T(1.0)});
  if (i == 3) p.t.push_back({{0, 0, 1, 0}, T(1.0)});
  if (i == 4) {
    p.t.push_back({{2, 0, 0, 0}, T(0.5)});
    p.t.push_back({{0, 2, 0, 0}, T(0.5)});
    p.t.push_back({{0, 0, 2, 0}, T(0.5)});
    p.t.push_back({{0, 0, 0, 1}, T(0.5)});
  }
  return p;
}
template <class T>
Poly<T> mul(const Poly<T>& a, const Poly<T>& b) {
  Poly<T> c;
  for (auto& x : a.t)
    for (auto& y : b.t) {
      std::array<int, 4> e;
      for (int k = 0; k < 4; ++k) e[k] = x.first[k] + y.first[k];
      c.t.push_back({e, x.second * y.second});
    }
  return c;
}
template <class T>
Poly<T> combo(const T* a) {  // sum_j a_j psi_j
  Poly<T> p;
  for (int j = 0; j < 5; ++j)
    for (auto& x : psi<T>(j).t) p.t.push_back({x.first, a[j] * x.second});
  return p;
}
template <class T>
Poly<T> add(const Poly<T>& a, const Poly<T>& b) {
  Poly<T> c = a;
  for (auto& x : b.t) c.t.push_back(x);
  return c;
}
template <class T>
Poly<T> mono(int a, int b, int c) {
  Poly<T> p;
  p.t.push_back({{a, b, c, 0}, T(1.0)});
  return p;
}

// Moments <u^a v^b w^c xi^(2d)> of a Maxwellian normalised to unit density.
template <class T>
struct Moments {
  T u[10], v[10], w[10], xi[3];
};
enum Range { kFull, kPos, kNeg };
template <class T>
Moments<T> moments(T U, T V, T W, T lam, double K, Range range) {
  Moments<T> M;
  auto full = [&](T c, T* out) {
    out[0] = T(1.0);
    out[1] = c;
    for (int n = 2; n < 10; ++n) out[n] = c * out[n - 1] + ((n - 1) / 2.0) * out[n - 2] / lam;
  };
  full(V, M.v);
  full(W, M.w);
  if (range == kFull) {
    full(U, M.u);
  } else {
    const double sg = range == kPos ? 1.0 : -1.0;
    M.u[0] = 0.5 * erfc(-sg * sqrt(lam) * U);
    M.u[1] = U * M.u[0] + sg * 0.5 * exp(-lam * U * U) / sqrt(M_PI * lam);
    for (int n = 2; n < 10; ++n) M.u[n] = U * M.u[n - 1] + ((n - 1) / 2.0) * M.u[n - 2] / lam;
  }
  M.xi[0] = T(1.0);
  M.xi[1] = K / (2.0 * lam);
  M.xi[2] = K * (K + 2.0) / (4.0 * lam * lam);
  return M;
}
template <class T>
T moment(const Poly<T>& p, const Moments<T>& M) {
  T s = T(0.0);
  for (auto& x : p.t) s += x.second * M.u[x.first[0]] * M.v[x.first[1]] * M.w[x.first[2]] * M.xi[x.first[3]];
  return s;
}
template <class T>
void moment_vec(const Poly<T>& p, const Moments<T>& M, T out[5]) {
  for (int i = 0; i < 5; ++i) out[i] = moment(mul(psi<T>(i), p), M);
}

template <class T>
struct Prim {
  T rho, U, V, W, lam, p;
};
template <class T>
bool primitive(const T* q, double gamma, Prim<T>& w) {
  w.rho = q[0];
  if (!(val(w.rho) > 0.0)) return false;
  w.U = q[1] / q[0];
  w.V = q[2] / q[0];
  w.W = q[3] / q[0];
  w.p = (gamma - 1.0) * (q[4] - 0.5 * w.rho * (w.U * w.U + w.V * w.V + w.W * w.W));
  if (!(val(w.p) > 0.0)) return false;
  w.lam = w.rho / (2.0 * w.p);
  return true;
}

// Microscopic slope: solve <a psi> = b (b already divided by rho) as a dense 5x5 system.
template <class T>
void slope(const Moments<T>& M, const T* b, T* a) {
  T A[5][5], rhs[5];
  for (int i = 0; i < 5; ++i) {
    for (int j = 0; j < 5; ++j) A[i][j] = moment(mul(psi<T>(i), psi<T>(j)), M);
    rhs[i] = b[i];
  }
  solve5(A, rhs, a);
}

// Time integrals over [0, delta] of the coefficients in Eq. flux-1:
// c1 (1-e), c2 ((t+tau)e - tau), c3 (t - tau + tau e), c4 e, c5 -(tau+t) e, c6 -tau e,
// with e = exp(-t/tau); tau = 0 gives the limits.
template <class T>
void time_coeffs(T tau, double d, T c[6]) {
  if (!(val(tau) > 0.0)) {
    c[0] = T(d);
    c[1] = T(0.0);
    c[2] = T(0.5 * d * d);
    c[3] = c[4] = c[5] = T(0.0);
    return;
  }
  const T e = exp(-d / tau);
  c[0] = d - tau * (1.0 - e);
  c[1] = 2.0 * tau * tau * (1.0 - e) - tau * d * (1.0 + e);
  c[2] = 0.5 * d * d - tau * d + tau * tau * (1.0 - e);
  c[3] = tau * (1.0 - e);
  c[4] = -2.0 * tau * tau * (1.0 - e) + tau * d * e;
  c[5] = -tau * tau * (1.0 - e);
}

// Dynamic viscosity at temperature T = p / rho: mu (T / T_ref)^mu_pow for the power law of
// Section 5.4 (collision-time model 3), mu otherwise.
template <class T>
T viscosity(const Params& P, T temp) {
  if (P.tau_model == 3) return P.mu * pow(temp / P.T_ref, P.mu_pow);
  return T(P.mu);
}

// Local-frame flux at one Gauss point. dq*[m][v] = derivative of conserved variable v along n_m.
// Outputs the time integrals F(dt/2) and F(dt). Returns false for a non-physical state.
template <class T>
bool gp_flux(const Params& P, const T ql[5], const T dql[3][5], const T qr[5], const T dqr[3][5],
             double dt, T F[2][5]) {
  const double K = (5.0 - 3.0 * P.gamma) / (P.gamma - 1.0);
  Prim<T> wl, wr, w0;
  if (!primitive(ql, P.gamma, wl) || !primitive(qr, P.gamma, wr)) return false;
  const Moments<T> Ml = moments(wl.U, wl.V, wl.W, wl.lam, K, kFull);
  const Moments<T> Mr = moments(wr.U, wr.V, wr.W, wr.lam, K, kFull);
  const Moments<T> Mlp = moments(wl.U, wl.V, wl.W, wl.lam, K, kPos);
  const Moments<T> Mrn = moments(wr.U, wr.V, wr.W, wr.lam, K, kNeg);
  // slopes of both sides in the three directions, and their time slopes A
  T al[3][5], ar[3][5], Al[5], Ar[5];
  for (int d = 0; d < 3; ++d) {
    T bl[5], br[5];
    for (int v = 0; v < 5; ++v) {
      bl[v] = dql[d][v] / wl.rho;
      br[v] = dqr[d][v] / wr.rho;
    }
    slope(Ml, bl, al[d]);
    slope(Mr, br, ar[d]);
  }
  auto a_dot_u = [&](T a3[3][5]) {  // a_1 u + a_2 v + a_3 w as a polynomial
    return add(add(mul(mono<T>(1, 0, 0), combo<T>(a3[0])), mul(mono<T>(0, 1, 0), combo<T>(a3[1]))),
               mul(mono<T>(0, 0, 1), combo<T>(a3[2])));
  };
  {
    T rl[5], rr[5];
    moment_vec(a_dot_u(al), Ml, rl);
    moment_vec(a_dot_u(ar), Mr, rr);
    for (int v = 0; v < 5; ++v) {
      rl[v] = -rl[v];
      rr[v] = -rr[v];
    }
    slope(Ml, rl, Al);
    slope(Mr, rr, Ar);
  }
  // interface equilibrium from the two half-space moments
  T q0[5], tl[5], tr[5];
  const Poly<T> one = mono<T>(0, 0, 0);
  moment_vec(one, Mlp, tl);
  moment_vec(one, Mrn, tr);
  for (int v = 0; v < 5; ++v) q0[v] = wl.rho * tl[v] + wr.rho * tr[v];
  if (!primitive(q0, P.gamma, w0)) return false;
  const Moments<T> M0 = moments(w0.U, w0.V, w0.W, w0.lam, K, kFull);
  T abar[3][5], Abar[5];
  for (int d = 0; d < 3; ++d) {
    T sl[5], sr[5], b[5];
    moment_vec(combo<T>(al[d]), Mlp, sl);
    moment_vec(combo<T>(ar[d]), Mrn, sr);
    for (int v = 0; v < 5; ++v) b[v] = (wl.rho * sl[v] + wr.rho * sr[v]) / w0.rho;
    slope(M0, b, abar[d]);
  }
  {
    T r0[5];
    moment_vec(a_dot_u(abar), M0, r0);
    for (int v = 0; v < 5; ++v) r0[v] = -r0[v];
    slope(M0, r0, Abar);
  }
  // collision time
  T tau = T(0.0);
  const T dp = fabs((wl.p - wr.p) / (wl.p + wr.p));
  if (P.tau_model == 1) tau = P.tau_eps * dt + P.tau_C * dp * dt;
  if (P.tau_model == 2) tau = P.mu / w0.p + P.tau_C * dp * dt;
  if (P.tau_model == 3) tau = viscosity(P, w0.p / w0.rho) / w0.p + P.tau_C * dp * dt;
  // flux moments
  const Poly<T> u1 = mono<T>(1, 0, 0);
  T e0[5], e1[5], e2[5], nl0[5], nl1[5], nl2[5], nr0[5], nr1[5], nr2[5];
  moment_vec(u1, M0, e0);
  moment_vec(mul(u1, a_dot_u(abar)), M0, e1);
  moment_vec(mul(u1, combo<T>(Abar)), M0, e2);
  moment_vec(u1, Mlp, nl0);
  moment_vec(mul(u1, a_dot_u(al)), Mlp, nl1);
  moment_vec(mul(u1, combo<T>(Al)), Mlp, nl2);
  moment_vec(u1, Mrn, nr0);
  moment_vec(mul(u1, a_dot_u(ar)), Mrn, nr1);
  moment_vec(mul(u1, combo<T>(Ar)), Mrn, nr2);
  const double deltas[2] = {0.5 * dt, dt};
  for (int s = 0; s < 2; ++s) {
    const double d = deltas[s];
    if (P.flux_mode == 1) {
      T c[6];
      time_coeffs(tau, d, c);
      for (int v = 0; v < 5; ++v)
        F[s][v] = w0.rho * (c[0] * e0[v] + c[1] * e1[v] + c[2] * e2[v]) +
                  wl.rho * (c[3] * nl0[v] + c[4] * nl1[v] + c[5] * nl2[v]) +
                  wr.rho * (c[3] * nr0[v] + c[4] * nr1[v] + c[5] * nr2[v]);
    } else {
      for (int v = 0; v < 5; ++v)
        F[s][v] = w0.rho * (d * e0[v] - tau * d * (e1[v] + e2[v]) + 0.5 * d * d * e2[v]);
      if (P.Pr != 1.0) {
        // Prandtl-number fix of the BGK model (Xu 2001): the energy flux gains (1/Pr - 1) q with
        // q = <(u - U0) ((u-U0)^2 + (v-V0)^2 + (w-W0)^2 + xi^2) / 2 f>, the heat flux of the
        // time-integrated distribution relative to the interface velocity U0.
        Poly<T> cu, heat;
        cu.t.push_back({{1, 0, 0, 0}, T(1.0)});
        cu.t.push_back({{0, 0, 0, 0}, -w0.U});
        Poly<T> cv, cw, xi2;
        cv.t.push_back({{0, 1, 0, 0}, T(1.0)});
        cv.t.push_back({{0, 0, 0, 0}, -w0.V});
        cw.t.push_back({{0, 0, 1, 0}, T(1.0)});
        cw.t.push_back({{0, 0, 0, 0}, -w0.W});
        xi2.t.push_back({{0, 0, 0, 1}, T(1.0)});
        const Poly<T> c2 = add(add(add(mul(cu, cu), mul(cv, cv)), mul(cw, cw)), xi2);
        heat = mul(cu, c2);
        for (auto& x : heat.t) x.second = 0.5 * x.second;
        // f integrated over [0, d]: g0 [d (1 - tau (a.u + A)) + d^2/2 A]
        const Poly<T> one = mono<T>(0, 0, 0);
        Poly<T> fpoly;
        for (auto& x : one.t) fpoly.t.push_back({x.first, T(d) * x.second});
        for (auto& x : add(a_dot_u(abar), combo<T>(Abar)).t)
          fpoly.t.push_back({x.first, -tau * d * x.second});
        for (auto& x : combo<T>(Abar).t) fpoly.t.push_back({x.first, 0.5 * d * d * x.second});
        const T q = w0.rho * moment(mul(heat, fpoly), M0);
        F[s][4] += (1.0 / P.Pr - 1.0) * q;
      }
    }
  }
  return true;
}

// Local orthonormal frame at a Gauss point: n1 the normal, n2 = n1 x e_k / |.| with e_k the
// axis least aligned with n1, n3 = n1 x n2.
void frame(const double* n1, double n2[3], double n3[3]) {
  int k = 0;
  for (int a = 1; a < 3; ++a)
    if (std::fabs(n1[a]) < std::fabs(n1[k])) k = a;
  double e[3] = {0, 0, 0};
  e[k] = 1.0;
  cross(n1, e, n2);
  const double l = std::sqrt(n2[0] * n2[0] + n2[1] * n2[1] + n2[2] * n2[2]);
  for (int a = 0; a < 3; ++a) n2[a] /= l;
  cross(n1, n2, n3);
}

// ---------------------------------------------------------------------------------------------
// Residual L(Q) and its time derivative (Eq. finite with the two-point time fit).
template <class T>
bool face_flux(const Mesh& m, const Params& P, const Face& fc, const Recon<T>& ro,
               const Recon<T>* rn, double dt, T* out);

template <class T>
int residual(const Mesh& m, const Params& P, const T* Q, double dt, T* Lo, T* Lto,
             std::string& err) {
  const int n = m.n_cells;
  std::vector<Recon<T>> rec(n);
  for (int i = 0; i < n; ++i) {
    Prim<T> w;
    T q[5];
    for (int v = 0; v < 5; ++v) q[v] = Q[v * (size_t)n + i];
    if (!primitive(q, P.gamma, w)) {
      err = "non-physical state in cell " + std::to_string(i);
      return ST_NONPHYS;
    }
  }
#pragma omp parallel for schedule(dynamic, 64)
  for (int i = 0; i < n; ++i) reconstruct_cell(m, P, Q, n, i, rec[i]);
  const int nf = (int)m.faces.size();
  std::vector<std::array<T, 10>> ff(nf);
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : bad)
  for (int f = 0; f < nf; ++f) {
    const Face& fc = m.faces[f];
    if (!face_flux(m, P, fc, rec[fc.owner], fc.nb >= 0 ? &rec[fc.nb] : nullptr, dt, ff[f].data()))
      ++bad;
  }
  if (bad) {
    err = "non-physical reconstructed state at a Gauss point";
    return ST_NONPHYS;
  }
  for (size_t k = 0; k < 5 * (size_t)n; ++k) Lo[k] = Lto[k] = T(0.0);
  for (int f = 0; f < nf; ++f) {
    const Face& fc = m.faces[f];
    for (int v = 0; v < 5; ++v) {
      Lo[v * (size_t)n + fc.owner] -= ff[f][v] / m.cells[fc.owner].vol;
      Lto[v * (size_t)n + fc.owner] -= ff[f][5 + v] / m.cells[fc.owner].vol;
      if (fc.nb >= 0) {
        Lo[v * (size_t)n + fc.nb] += ff[f][v] / m.cells[fc.nb].vol;
        Lto[v * (size_t)n + fc.nb] += ff[f][5 + v] / m.cells[fc.nb].vol;
      }
    }
  }
  return ST_OK;
}

// Far-field state at a boundary plane of outward unit normal n (Section 5.4: inlet and outlet
// by Riemann invariants). From the interior state q and the plane's far field, the invariants
// along n
// R+ = u_n + 2c/(gamma-1) (carried out of the domain) and R- = u_n - 2c/(gamma-1) (carried in)
// are taken from the interior and the far field; the boundary u_n and c are their mean and
// (gamma-1)/4 of their difference; the entropy p/rho^gamma and the tangential velocity come from
// the side the flow comes from. Supersonic inflow takes the far field, supersonic outflow the
// interior. Returns the conserved boundary state.
template <class T>
void farfield_state(const Params& P, int plane, const T* q, const double n[3], T* out) {
  const double g = P.gamma, gm1 = g - 1.0;
  const T rho = q[0];
  T U[3], un = T(0.0), ke = T(0.0);
  for (int a = 0; a < 3; ++a) {
    U[a] = q[1 + a] / rho;
    un += U[a] * n[a];
    ke += U[a] * U[a];
  }
  const T p = gm1 * (q[4] - 0.5 * rho * ke);
  const T c = sqrt(g * p / rho);
  const double rinf = P.finf[plane][0], pinf = P.finf[plane][4];
  const double* Uinf = P.finf[plane] + 1;
  double uninf = 0;
  for (int a = 0; a < 3; ++a) uninf += Uinf[a] * n[a];
  const double cinf = std::sqrt(g * pinf / rinf);
  auto set_prim = [&](T r, const T* V, T pr) {
    out[0] = r;
    T k = T(0.0);
    for (int a = 0; a < 3; ++a) {
      out[1 + a] = r * V[a];
      k += V[a] * V[a];
    }
    out[4] = pr / gm1 + 0.5 * r * k;
  };
  if (val(un) >= val(c)) {  // supersonic outflow: everything from the interior
    for (int v = 0; v < 5; ++v) out[v] = q[v];
    return;
  }
  if (val(un) <= -val(c)) {  // supersonic inflow: everything from the far field
    T V[3] = {T(Uinf[0]), T(Uinf[1]), T(Uinf[2])};
    set_prim(T(rinf), V, T(pinf));
    return;
  }
  const T Rp = un + 2.0 * c / gm1;
  const T Rm = uninf - 2.0 * cinf / gm1;
  const T unb = 0.5 * (Rp + Rm);
  const T cb = 0.25 * gm1 * (Rp - Rm);
  T s, Vt[3];
  if (val(unb) >= 0.0) {  // outflow: entropy and tangential velocity of the interior
    s = p / pow(rho, g);
    for (int a = 0; a < 3; ++a) Vt[a] = U[a] - un * n[a];
  } else {
    s = T(pinf / std::pow(rinf, g));
    for (int a = 0; a < 3; ++a) Vt[a] = T(Uinf[a] - uninf * n[a]);
  }
  const T rb = pow(cb * cb / (g * s), 1.0 / gm1);
  const T pb = rb * cb * cb / g;
  T V[3];
  for (int a = 0; a < 3; ++a) V[a] = Vt[a] + unb * n[a];
  set_prim(rb, V, pb);
}

// Ghost state at a wall point (Section 2: the ghost's flow variables follow the boundary
// condition; the paper names slip, no-slip adiabatic and no-slip isothermal walls in Section 5
// and gives no formulas). From the owner's value v and gradient g at the point (global frame),
// the image across the plane of axis a: geometry mirrored, so d/dx_a changes sign, and
//   slip:               the normal momentum negated;
//   no-slip (U_w, T_w): rho_g = rho, U_g = 2 U_w - U, and
//     adiabatic (T_w <= 0): p_g = p, i.e. E_g = E + 2 rho |U_w|^2 - 2 U_w . m,
//     isothermal:           T_g = 2 T_w - T with T = p / rho, i.e.
//                           E_g = 2 rho T_w / (gamma-1) - E + |m|^2/rho + 2 rho |U_w|^2 - 2 U_w . m.
// The ghost gradient is the mirrored gradient mapped by the Jacobian of that map at v.
template <class T>
void wall_ghost(const Params& P, int kind, int plane, const T* v, const T g[5][3], T* vg,
                T gg[5][3]) {
  const int ax = plane % 3;
  if (kind == 3) {  // far field: the characteristic boundary state, uniform (no gradient)
    double n[3] = {0, 0, 0};
    n[ax] = plane >= 3 ? 1.0 : -1.0;
    farfield_state(P, plane, v, n, vg);
    for (int r = 0; r < 5; ++r)
      for (int b = 0; b < 3; ++b) gg[r][b] = T(0.0);
    return;
  }
  T J[5][5];
  for (int r = 0; r < 5; ++r)
    for (int c = 0; c < 5; ++c) J[r][c] = T(r == c ? 1.0 : 0.0);
  if (kind == 1) {
    J[1 + ax][1 + ax] = T(-1.0);
    for (int r = 0; r < 5; ++r) vg[r] = v[r];
    vg[1 + ax] = -v[1 + ax];
  } else {
    const double* uw = P.uw[plane];
    const double Tw = P.Tw[plane];
    const double uw2 = uw[0] * uw[0] + uw[1] * uw[1] + uw[2] * uw[2];
    const T rho = v[0];
    T um = T(0.0);
    for (int a = 0; a < 3; ++a) um += uw[a] * v[1 + a];
    vg[0] = rho;
    for (int a = 0; a < 3; ++a) {
      vg[1 + a] = 2.0 * uw[a] * rho - v[1 + a];
      J[1 + a][0] = T(2.0 * uw[a]);
      J[1 + a][1 + a] = T(-1.0);
    }
    if (Tw <= 0.0) {
      vg[4] = v[4] + 2.0 * uw2 * rho - 2.0 * um;
      J[4][0] = T(2.0 * uw2);
      for (int a = 0; a < 3; ++a) J[4][1 + a] = T(-2.0 * uw[a]);
    } else {
      T m2 = T(0.0);
      for (int a = 0; a < 3; ++a) m2 += v[1 + a] * v[1 + a];
      const T U2 = m2 / (rho * rho);
      vg[4] = 2.0 * Tw / (P.gamma - 1.0) * rho - v[4] + m2 / rho + 2.0 * uw2 * rho - 2.0 * um;
      J[4][0] = 2.0 * Tw / (P.gamma - 1.0) - U2 + 2.0 * uw2;
      for (int a = 0; a < 3; ++a) J[4][1 + a] = 2.0 * v[1 + a] / rho - 2.0 * uw[a];
      J[4][4] = T(-1.0);
    }
  }
  for (int r = 0; r < 5; ++r)
    for (int b = 0; b < 3; ++b) {
      T x = T(0.0);
      for (int c = 0; c < 5; ++c) x += J[r][c] * g[c][b];
      gg[r][b] = b == ax ? -x : x;
    }
}

// Positivity fallback at one Gauss point (a reading, not in the paper, which prints no
// positivity treatment): when the reconstructed state of a side has rho <= 0 or p <= 0 (or is
// NaN), that side takes its cell average and a zero gradient, the first-order state.
template <class T>
bool physical_state(const T q[5]) {
  // p > 0 written as rho E > |m|^2 / 2 (rho > 0): the form the decision takes on both sides
  const double r = val(q[0]);
  const double m2 = val(q[1]) * val(q[1]) + val(q[2]) * val(q[2]) + val(q[3]) * val(q[3]);
  return r > 0.0 && r * val(q[4]) > 0.5 * m2;
}
template <class T>
void gp_first_order(const Recon<T>& r, T v[5], T g[5][3]) {
  if (physical_state(v)) return;
  for (int c = 0; c < 5; ++c) {
    v[c] = r.Q0[c];
    for (int a = 0; a < 3; ++a) g[c][a] = T(0.0);
  }
}

// Face flux (Eq. flux-qud over the 2x2 Gauss points) fitted in time:
// out[0..4] = F^n, out[5..9] = dF/dt. Returns false for a non-physical state.
template <class T>
bool face_flux(const Mesh& m, const Params& P, const Face& fc, const Recon<T>& ro,
               const Recon<T>* rn, double dt, T* out) {
  {
    T acc[2][5];
    for (int s = 0; s < 2; ++s)
      for (int v = 0; v < 5; ++v) acc[s][v] = T(0.0);
    for (int k = 0; k < 4; ++k) {
      T vl[5], gl[5][3], vr[5], gr[5][3];
      eval_recon(m, fc.owner, ro, fc.xg[k], vl, gl);
      if (P.gp_fallback) gp_first_order(ro, vl, gl);
      if (fc.nb >= 0) {
        double xn[3];
        for (int a = 0; a < 3; ++a) xn[a] = (fc.xg[k][a] - fc.nb_to_owner.t[a]) / fc.nb_to_owner.s[a];
        T v0[5], g0[5][3];
        eval_recon(m, fc.nb, *rn, xn, v0, g0);
        if (P.gp_fallback) gp_first_order(*rn, v0, g0);
        transform_state(m, P, fc.nb_to_owner, v0, vr);
        for (int v = 0; v < 5; ++v) {
          const double sv = (v >= 1 && v <= 3 && ((fc.nb_to_owner.vflip >> (v - 1)) & 1)) ? -1.0 : 1.0;
          for (int a = 0; a < 3; ++a) gr[v][a] = sv * fc.nb_to_owner.s[a] * g0[v][a];
        }
      } else {
        // the wall's ghost at the Gauss point
        wall_ghost(P, fc.wall_kind, fc.wall_plane, vl, gl, vr, gr);
      }
      // rotate into the local frame
      const double* n1 = fc.n[k];
      double n2[3], n3[3];
      frame(n1, n2, n3);
      const double* nm[3] = {n1, n2, n3};
      auto rot = [&](const T* q, T* out) {
        out[0] = q[0];
        for (int d = 0; d < 3; ++d) out[1 + d] = q[1] * nm[d][0] + q[2] * nm[d][1] + q[3] * nm[d][2];
        out[4] = q[4];
      };
      T ql[5], qr[5], dql[3][5], dqr[3][5];
      rot(vl, ql);
      rot(vr, qr);
      for (int d = 0; d < 3; ++d) {
        T sl[5], sr[5];
        for (int v = 0; v < 5; ++v) {
          sl[v] = gl[v][0] * nm[d][0] + gl[v][1] * nm[d][1] + gl[v][2] * nm[d][2];
          sr[v] = gr[v][0] * nm[d][0] + gr[v][1] * nm[d][1] + gr[v][2] * nm[d][2];
        }
        rot(sl, dql[d]);
        rot(sr, dqr[d]);
      }
      T F[2][5];
      if (!gp_flux(P, ql, dql, qr, dqr, dt, F)) return false;
      for (int s = 0; s < 2; ++s) {
        T g[5];
        g[0] = F[s][0];
        for (int a = 0; a < 3; ++a) g[1 + a] = F[s][1] * n1[a] + F[s][2] * n2[a] + F[s][3] * n3[a];
        g[4] = F[s][4];
        for (int v = 0; v < 5; ++v) acc[s][v] += fc.w[k] * g[v];
      }
    }
    if (fc.nb < 0 && fc.wall_kind != 3) {
      // walls are impermeable: no mass flux. A slip wall passes only normal momentum (its
      // exact flux by symmetry); an adiabatic no-slip wall conducts no heat, so its energy flux
      // is the work of the wall force, U_w . F_m; an isothermal wall keeps the GKS energy flux
      for (int s = 0; s < 2; ++s) {
        acc[s][0] = T(0.0);
        if (fc.wall_kind == 1) {
          for (int v = 1; v < 5; ++v)
            if (v != 1 + fc.wall_axis) acc[s][v] = T(0.0);
        } else if (P.Tw[fc.wall_plane] <= 0.0) {
          const double* uw = P.uw[fc.wall_plane];
          acc[s][4] = uw[0] * acc[s][1] + uw[1] * acc[s][2] + uw[2] * acc[s][3];
        }
      }
    }
    for (int v = 0; v < 5; ++v) {
      out[v] = (4.0 * acc[0][v] - acc[1][v]) / dt;
      out[5 + v] = 4.0 * (acc[1][v] - 2.0 * acc[0][v]) / (dt * dt);
    }
  }
  return true;
}

// Two-stage fourth-order update (Section 3.3).
template <class T>
void s2o4_stage1(size_t len, const T* Q, const T* L, const T* Lt, double dt, T* Qs) {
  for (size_t k = 0; k < len; ++k) Qs[k] = Q[k] + 0.5 * dt * L[k] + (dt * dt / 8.0) * Lt[k];
}
template <class T>
void s2o4_stage2(size_t len, const T* Q, const T* L, const T* Lt, const T* Lts, double dt, T* Qn) {
  for (size_t k = 0; k < len; ++k) Qn[k] = Q[k] + dt * L[k] + (dt * dt / 6.0) * (Lt[k] + 2.0 * Lts[k]);
}
template <class T>
int step(const Mesh& m, const Params& P, T* Q, double dt, int nsteps, std::string& err) {
  const size_t len = 5 * (size_t)m.n_cells;
  std::vector<T> L(len), Lt(len), Qs(len), Ls(len), Lts(len);
  for (int s = 0; s < nsteps; ++s) {
    int st = residual(m, P, Q, dt, L.data(), Lt.data(), err);
    if (st) return st;
    s2o4_stage1(len, Q, L.data(), Lt.data(), dt, Qs.data());
    st = residual(m, P, Qs.data(), dt, Ls.data(), Lts.data(), err);
    if (st) return st;
    s2o4_stage2(len, Q, L.data(), Lt.data(), Lts.data(), dt, Q);
  }
  return ST_OK;
}

// ---------------------------------------------------------------------------------------------
// Implicit step (Section 4): backward Euler with the residual's change linearised by the flux
// splitting F = (T(Q_i) + T(Q_p) - r (Q_p - Q_i))/2 . n S, the resulting system
//   (|Omega_i|/dt + 1/2 sum_f r_f S_f) dQ_i + 1/2 sum_f [T_n(Q_p + dQ_p) - T_n(Q_p) - r_f dQ_p] S_f
//     = |Omega_i| Res_i
// solved by kmax Jacobi iterations from dQ^(0) = |Omega_i| Res_i / D_i. Res_i is the GKS residual
// averaged over [0, dt]: Res = L + dt/2 Lt (the time integral of the fitted face flux over the
// step). T_n(Q) = T(Q) . n is the Euler flux through the face with n pointing out of cell i,
// S_f the face area and r_f = max over the two sides of |U . n| + c at Q^n. A wall face couples
// the cell to its mirror image.
double sound_speed_normal(const double* q, const double n[3], double gamma) {
  const double U[3] = {q[1] / q[0], q[2] / q[0], q[3] / q[0]};
  const double p = (gamma - 1.0) * (q[4] - 0.5 * q[0] * (U[0] * U[0] + U[1] * U[1] + U[2] * U[2]));
  return std::fabs(U[0] * n[0] + U[1] * n[1] + U[2] * n[2]) + std::sqrt(gamma * p / q[0]);
}
void euler_normal_flux(const double* q, const double n[3], double gamma, double* T) {
  const double U[3] = {q[1] / q[0], q[2] / q[0], q[3] / q[0]};
  const double p = (gamma - 1.0) * (q[4] - 0.5 * q[0] * (U[0] * U[0] + U[1] * U[1] + U[2] * U[2]));
  const double un = U[0] * n[0] + U[1] * n[1] + U[2] * n[2];
  T[0] = q[0] * un;
  for (int a = 0; a < 3; ++a) T[1 + a] = q[1 + a] * un + p * n[a];
  T[4] = (q[4] + p) * un;
}

int step_implicit(const Mesh& m, const Params& P, double* Q, double dt, int nsteps, int kmax,
                  std::string& err) {
  const int n = m.n_cells, nf = (int)m.faces.size();
  const size_t len = 5 * (size_t)n;
  // per face: area vector sum_k w_k n_k (out of the owner) and area
  std::vector<std::array<double, 3>> nrm(nf);
  std::vector<double> area(nf);
  for (int f = 0; f < nf; ++f) {
    double a[3] = {0, 0, 0};
    for (int k = 0; k < 4; ++k)
      for (int c = 0; c < 3; ++c) a[c] += m.faces[f].w[k] * m.faces[f].n[k][c];
    area[f] = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    for (int c = 0; c < 3; ++c) nrm[f][c] = a[c] / area[f];
  }
  std::vector<double> L(len), Lt(len), R(len), D(n), dQ(len), dQn(len);
  auto get = [&](const double* X, int i, double* q) {
    for (int v = 0; v < 5; ++v) q[v] = X[v * (size_t)n + i];
  };
  // the other side of face f seen from cell i: state and increment in cell i's frame, the
  // unit normal out of cell i
  auto other = [&](int f, int i, const double* X, const double* dX, double* qp, double* dqp,
                   double nn[3]) {
    const Face& fc = m.faces[f];
    const bool own = fc.owner == i;
    for (int c = 0; c < 3; ++c) nn[c] = own ? nrm[f][c] : -nrm[f][c];
    double q[5], dq[5];
    if (fc.nb < 0) {  // the wall's ghost of the cell: Q_p = G(Q_i), dQ_p = G(Q_i + dQ_i) - G(Q_i)
      get(X, i, q);
      get(dX, i, dq);
      double zg[5][3] = {}, zgg[5][3];
      wall_ghost(P, fc.wall_kind, fc.wall_plane, q, zg, qp, zgg);
      if (fc.wall_kind == 3) {  // far field: the change of the characteristic state
        double q1[5], g1[5];
        for (int v = 0; v < 5; ++v) q1[v] = q[v] + dq[v];
        wall_ghost(P, fc.wall_kind, fc.wall_plane, q1, zg, g1, zgg);
        for (int v = 0; v < 5; ++v) dqp[v] = g1[v] - qp[v];
        return;
      }
      // the slip and adiabatic maps are linear: dQ_p = G(dQ_i)
      wall_ghost(P, fc.wall_kind, fc.wall_plane, dq, zg, dqp, zgg);
      if (fc.wall_kind == 2 && P.Tw[fc.wall_plane] > 0.0) {
        // isothermal: the change of |m|^2/rho written without cancellation,
        // (2 m . dm + |dm|^2 - |m|^2 drho / rho) / (rho + drho)
        const double r = q[0], dr = dq[0];
        const double* uw = P.uw[fc.wall_plane];
        double mdm = 0, dm2 = 0, m2 = 0, uwdm = 0;
        for (int a = 0; a < 3; ++a) {
          mdm += q[1 + a] * dq[1 + a];
          dm2 += dq[1 + a] * dq[1 + a];
          m2 += q[1 + a] * q[1 + a];
          uwdm += uw[a] * dq[1 + a];
        }
        const double uw2 = uw[0] * uw[0] + uw[1] * uw[1] + uw[2] * uw[2];
        dqp[4] = (2.0 * P.Tw[fc.wall_plane] / (P.gamma - 1.0) + 2.0 * uw2) * dr - dq[4] +
                 (2.0 * mdm + dm2 - m2 * dr / r) / (r + dr) - 2.0 * uwdm;
      }
      return;
    }
    const int p = own ? fc.nb : fc.owner;
    get(X, p, q);
    get(dX, p, dq);
    // periodic images are translations: the state is the same in both frames
    for (int v = 0; v < 5; ++v) {
      qp[v] = q[v];
      dqp[v] = dq[v];
    }
  };
  for (int s = 0; s < nsteps; ++s) {
    int st = residual(m, P, Q, dt, L.data(), Lt.data(), err);
    if (st) return st;
    for (int i = 0; i < n; ++i) {
      double sum = 0.0, qi[5];
      get(Q, i, qi);
      for (int f : m.cells[i].face_id) {
        double qp[5], dqp[5], nn[3];
        other(f, i, Q, Q, qp, dqp, nn);
        const double r = std::max(sound_speed_normal(qi, nn, P.gamma),
                                  sound_speed_normal(qp, nn, P.gamma));
        sum += 0.5 * r * area[f];
      }
      D[i] = m.cells[i].vol / dt + sum;
      for (int v = 0; v < 5; ++v) {
        const size_t k = v * (size_t)n + i;
        R[k] = m.cells[i].vol * (L[k] + 0.5 * dt * Lt[k]);
        dQ[k] = R[k] / D[i];
      }
    }
    for (int it = 0; it < kmax; ++it) {
      for (int i = 0; i < n; ++i) {
        double acc[5] = {0, 0, 0, 0, 0}, qi[5];
        get(Q, i, qi);
        for (int f : m.cells[i].face_id) {
          double qp[5], dqp[5], nn[3], q1[5], T0[5], T1[5];
          other(f, i, Q, dQ.data(), qp, dqp, nn);
          const double r = std::max(sound_speed_normal(qi, nn, P.gamma),
                                    sound_speed_normal(qp, nn, P.gamma));
          for (int v = 0; v < 5; ++v) q1[v] = qp[v] + dqp[v];
          euler_normal_flux(q1, nn, P.gamma, T1);
          euler_normal_flux(qp, nn, P.gamma, T0);
          for (int v = 0; v < 5; ++v) acc[v] += 0.5 * (T1[v] - T0[v] - r * dqp[v]) * area[f];
        }
        for (int v = 0; v < 5; ++v) {
          const size_t k = v * (size_t)n + i;
          dQn[k] = (R[k] - acc[v]) / D[i];
        }
      }
      std::swap(dQ, dQn);
    }
    for (size_t k = 0; k < len; ++k) Q[k] += dQ[k];
    for (int i = 0; i < n; ++i) {
      double q[5];
      Prim<double> w;
      get(Q, i, q);
      if (!primitive(q, P.gamma, w)) {
        err = "non-physical state after the implicit update in cell " + std::to_string(i);
        return ST_NONPHYS;
      }
    }
  }
  return ST_OK;
}

}  // namespace

// =============================================================================================
// C entry points (used through ctypes by the tests).
extern "C" {

// lazy != 0 builds only topology and geometry; stencils are built on first use (for the
// sampled residual on large meshes).
void* oracle_mesh_create(int64_t n_nodes, const double* xyz, int64_t n_cells,
                         const int8_t* cell_type, const int64_t* cell_nodes, const int* bc,
                         const double* lo, const double* hi, int lazy, int min_stencil,
                         int* status, char* errbuf, int errlen) {
  Mesh* m = new Mesh;
  m->min_stencil = min_stencil;
  m->n_nodes = (int)n_nodes;
  m->n_cells = (int)n_cells;
  m->xyz.assign(xyz, xyz + 3 * n_nodes);
  for (int a = 0; a < 3; ++a) {
    m->bc[a] = bc[a];
    m->lo[a] = lo[a];
    m->hi[a] = hi[a];
    m->L[a] = hi[a] - lo[a];
  }
  m->cells.resize(n_cells);
  for (int64_t c = 0; c < n_cells; ++c) {
    m->cells[c].type = cell_type[c];
    for (int s = 0; s < 8; ++s) m->cells[c].node[s] = (int)cell_nodes[8 * c + s];
  }
  *status = build_mesh(*m, lazy != 0);
  if (*status) {
    if (errbuf && errlen > 0) {
      std::strncpy(errbuf, m->err.c_str(), errlen - 1);
      errbuf[errlen - 1] = 0;
    }
    delete m;
    return nullptr;
  }
  return m;
}

void oracle_mesh_destroy(void* h) { delete static_cast<Mesh*>(h); }

int64_t oracle_n_faces(void* h) { return (int64_t) static_cast<Mesh*>(h)->faces.size(); }

// Conditioning of each cell's big-stencil least-squares matrix: max |R_jj| / min |R_jj| of its
// Householder factor (a lower bound of the 2-norm condition number).
void oracle_stencil_conditioning(void* h, double* out) {
  Mesh* m = static_cast<Mesh*>(h);
  for (int i = 0; i < m->n_cells; ++i) {
    build_cell_stencil(*m, i);
    double lo = 1e300, hi = 0;
    for (double r : m->cells[i].qr0.rdiag) {
      lo = std::min(lo, std::fabs(r));
      hi = std::max(hi, std::fabs(r));
    }
    out[i] = m->cells[i].qr0.rdiag.empty() ? 0.0 : hi / lo;
  }
}

// vol[n], centroid[n][3], K[n] stencil size, M[n] sub-stencil count, plain[n] (1 if no member
// carries a periodic or mirror transform)
void oracle_cell_info(void* h, double* vol, double* centroid, int* K, int* M, int* plain) {
  Mesh* m = static_cast<Mesh*>(h);
  for (int i = 0; i < m->n_cells; ++i) {
    const Cell& c = m->cells[i];
    vol[i] = c.vol;
    for (int a = 0; a < 3; ++a) centroid[3 * i + a] = c.centroid[a];
    K[i] = (int)c.stencil.size();
    M[i] = (int)c.sub.size();
    plain[i] = c.plain ? 1 : 0;
  }
}

// owner[nf], nb[nf] (-1 wall), shift[nf][3], xg[nf][4][3], normal[nf][4][3], w[nf][4]
void oracle_face_info(void* h, int* owner, int* nb, double* shift, double* xg, double* nrm,
                      double* w) {
  Mesh* m = static_cast<Mesh*>(h);
  for (size_t f = 0; f < m->faces.size(); ++f) {
    const Face& fc = m->faces[f];
    owner[f] = fc.owner;
    nb[f] = fc.nb;
    for (int a = 0; a < 3; ++a) shift[3 * f + a] = fc.nb >= 0 ? fc.nb_to_owner.t[a] : 0.0;
    for (int k = 0; k < 4; ++k) {
      for (int a = 0; a < 3; ++a) {
        xg[12 * f + 3 * k + a] = fc.xg[k][a];
        nrm[12 * f + 3 * k + a] = fc.n[k][a];
      }
      w[4 * f + k] = fc.w[k];
    }
  }
}

// Exact (27-point) cell averages of a field. field 0: the advected density sine wave at time t
// (Section 5.1)
// (gamma = fp[0]); field 1: a quadratic per conserved variable, fp = [5][10] coefficients of
// (1, x, y, z, xx, yy, zz, xy, xz, yz).
int oracle_cell_average(void* h, int field, double t, const double* fp, double* Q) {
  Mesh* m = static_cast<Mesh*>(h);
  const int n = m->n_cells;
  for (int i = 0; i < n; ++i) {
    const Quad27 q = quad27(m->cells[i].X);
    double acc[5] = {0, 0, 0, 0, 0}, vol = 0;
    for (int g = 0; g < 27; ++g) {
      const double* x = q.x[g];
      double val[5];
      if (field == 0) {
        const double gamma = fp[0];
        // the profile moves with the velocity (1,1,1): x + y + z - 3t (Section 5.1 prints
        // x + y + z - t, which agrees with this only when t is a multiple of 2/3)
        const double rho = 1.0 + 0.2 * std::sin(M_PI * (x[0] + x[1] + x[2] - 3.0 * t));
        val[0] = rho;
        val[1] = val[2] = val[3] = rho;
        val[4] = 1.0 / (gamma - 1.0) + 0.5 * rho * 3.0;
      } else if (field == 1) {
        const double mono[10] = {1, x[0], x[1], x[2], x[0] * x[0], x[1] * x[1], x[2] * x[2],
                                 x[0] * x[1], x[0] * x[2], x[1] * x[2]};
        for (int v = 0; v < 5; ++v) {
          val[v] = 0;
          for (int k = 0; k < 10; ++k) val[v] += fp[10 * v + k] * mono[k];
        }
      } else {
        return ST_INVAL;
      }
      vol += q.w[g];
      for (int v = 0; v < 5; ++v) acc[v] += q.w[g] * val[v];
    }
    for (int v = 0; v < 5; ++v) Q[v * (size_t)n + i] = acc[v] / vol;
  }
  return ST_OK;
}

// Reconstructed values and gradients at points inside (or on the boundary of) given cells.
// out[p][5][4] = (value, d/dx, d/dy, d/dz) per conserved variable.
int oracle_reconstruct_at(void* h, const double* params, const double* Q, int npts,
                          const int* cell, const double* x, double* out) {
  Mesh* m = static_cast<Mesh*>(h);
  const Params P = read_params(params);
  for (int p = 0; p < npts; ++p) {
    Recon<double> r;
    reconstruct_cell(*m, P, Q, m->n_cells, cell[p], r);
    double v[5], g[5][3];
    eval_recon(*m, cell[p], r, x + 3 * p, v, g);
    for (int k = 0; k < 5; ++k) {
      out[20 * p + 4 * k] = v[k];
      for (int a = 0; a < 3; ++a) out[20 * p + 4 * k + 1 + a] = g[k][a];
    }
  }
  return ST_OK;
}

// The parts of one cell's reconstruction (Section 2), per conserved variable v: a[v][9] the
// coefficients of P0 in the scaled basis (x, y, z, xx, yy, zz, xy, xz, yz about the centroid,
// divided by h = |Omega|^(1/3) per power), b[v][M][3] those of the linear candidates, beta[v][M+1]
// and wbar[v][M+1] the indicators and normalised weights, tau[v]. Arrays are sized for M <= 16;
// *M_out and *h_out return M and h.
int oracle_weno_detail(void* h, const double* params, const double* Q, int cell, double* a,
                       double* b, double* beta, double* wbar, double* tau, int* M_out,
                       double* h_out) {
  Mesh* m = static_cast<Mesh*>(h);
  const Params P = read_params(params);
  if (cell < 0 || cell >= m->n_cells) return ST_INVAL;
  Recon<double> r;
  reconstruct_cell(*m, P, Q, m->n_cells, cell, r);
  *M_out = r.M;
  *h_out = m->cells[cell].h;
  for (int v = 0; v < 5; ++v) {
    for (int k = 0; k < 9; ++k) a[9 * v + k] = r.a[v][k];
    for (int s = 0; s < r.M; ++s)
      for (int k = 0; k < 3; ++k) b[(v * 16 + s) * 3 + k] = r.b[v][s][k];
    for (int s = 0; s <= r.M; ++s) {
      beta[17 * v + s] = r.beta[v][s];
      wbar[17 * v + s] = r.wbar[v][s];
    }
    tau[v] = r.tau[v];
  }
  return ST_OK;
}

// OpenMP threads of the oracle's loops over cells and faces (for timing it on 1 core and on
// all cores).
void oracle_set_threads(int n) { omp_set_num_threads(n > 0 ? n : 1); }
int oracle_max_threads() { return omp_get_max_threads(); }

// The nonlinear weights alone, from given indicators beta[0..M]: wbar[0..M]; returns tau.
double oracle_weno_weights(const double* params, int M, const double* beta, double* wbar) {
  const Params P = read_params(params);
  return nonlinear_weights(P, M, beta, wbar);
}

// One Gauss-point flux in the local frame: F[2][5] = time integrals over [0, dt/2], [0, dt].
int oracle_gp_flux(const double* params, const double* ql, const double* dql, const double* qr,
                   const double* dqr, double dt, double* F) {
  const Params P = read_params(params);
  double a[5], b[5], da[3][5], db[3][5], out[2][5];
  for (int v = 0; v < 5; ++v) {
    a[v] = ql[v];
    b[v] = qr[v];
    for (int d = 0; d < 3; ++d) {
      da[d][v] = dql[5 * d + v];
      db[d][v] = dqr[5 * d + v];
    }
  }
  if (!gp_flux(P, a, da, b, db, dt, out)) return ST_NONPHYS;
  for (int s = 0; s < 2; ++s)
    for (int v = 0; v < 5; ++v) F[5 * s + v] = out[s][v];
  return ST_OK;
}

void oracle_time_coeffs(double tau, double delta, double* c) { time_coeffs(tau, delta, c); }

// Ghost value and gradient at a wall point (global frame), g and gg as [5][3].
void oracle_wall_ghost(const double* params, int kind, int plane, const double* v,
                       const double* g, double* vg, double* gg) {
  const Params P = read_params(params);
  double G[5][3], GG[5][3];
  for (int r = 0; r < 5; ++r)
    for (int b = 0; b < 3; ++b) G[r][b] = g[3 * r + b];
  wall_ghost(P, kind, plane, v, G, vg, GG);
  for (int r = 0; r < 5; ++r)
    for (int b = 0; b < 3; ++b) gg[3 * r + b] = GG[r][b];
}

// Slope a (5) of <a psi> = b for a Maxwellian with primitive (U,V,W,lambda).
void oracle_slope(double U, double V, double W, double lam, double K, const double* b, double* a) {
  slope(moments(U, V, W, lam, K, kFull), b, a);
}

int oracle_residual(void* h, const double* params, const double* Q, double dt, double* L,
                    double* Lt, char* errbuf, int errlen) {
  Mesh* m = static_cast<Mesh*>(h);
  std::string err;
  const int st = residual(*m, read_params(params), Q, dt, L, Lt, err);
  if (st && errbuf && errlen > 0) {
    std::strncpy(errbuf, err.c_str(), errlen - 1);
    errbuf[errlen - 1] = 0;
  }
  return st;
}

// Directional derivative of the residual: (dL, dLt) = d(L, Lt)/dQ . dQ by forward dual numbers.
int oracle_residual_jvp(void* h, const double* params, const double* Q, const double* dQ,
                        double dt, double* L, double* Lt, double* dL, double* dLt) {
  Mesh* m = static_cast<Mesh*>(h);
  const size_t len = 5 * (size_t)m->n_cells;
  std::vector<Dual> q(len), l(len), lt(len);
  for (size_t k = 0; k < len; ++k) q[k] = Dual(Q[k], dQ[k]);
  std::string err;
  const int st = residual(*m, read_params(params), q.data(), dt, l.data(), lt.data(), err);
  if (st) return st;
  for (size_t k = 0; k < len; ++k) {
    L[k] = l[k].v;
    dL[k] = l[k].d;
    Lt[k] = lt[k].v;
    dLt[k] = lt[k].d;
  }
  return ST_OK;
}

// L and Lt of the listed cells only (out[p][5] each), for spot checks on large meshes.
int oracle_residual_cells(void* h, const double* params, const double* Q, double dt, int ncells,
                          const int* cells, double* L, double* Lt) {
  Mesh* m = static_cast<Mesh*>(h);
  const Params P = read_params(params);
  const int n = m->n_cells;
  std::map<int, Recon<double>> rec;
  auto get = [&](int c) -> const Recon<double>& {
    auto it = rec.find(c);
    if (it != rec.end()) return it->second;
    Recon<double>& r = rec[c];
    reconstruct_cell(*m, P, Q, n, c, r);
    return r;
  };
  for (int p = 0; p < ncells; ++p) {
    const int i = cells[p];
    if (i < 0 || i >= n) return ST_INVAL;
    std::vector<int> need = {i};
    for (int f : m->cells[i].face_id) {
      need.push_back(m->faces[f].owner);
      if (m->faces[f].nb >= 0) need.push_back(m->faces[f].nb);
    }
    for (int c : need) {
      const int st = build_cell_stencil(*m, c);
      if (st) return st;
    }
    double acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int f : m->cells[i].face_id) {
      const Face& fc = m->faces[f];
      double ff[10];
      const Recon<double>& ro = get(fc.owner);
      const Recon<double>* rn = fc.nb >= 0 ? &get(fc.nb) : nullptr;
      if (!face_flux(*m, P, fc, ro, rn, dt, ff)) return ST_NONPHYS;
      if (fc.owner == i)
        for (int v = 0; v < 10; ++v) acc[v] -= ff[v];
      if (fc.nb == i)
        for (int v = 0; v < 10; ++v) acc[v] += ff[v];
    }
    for (int v = 0; v < 5; ++v) {
      L[5 * p + v] = acc[v] / m->cells[i].vol;
      Lt[5 * p + v] = acc[5 + v] / m->cells[i].vol;
    }
  }
  return ST_OK;
}

int oracle_step(void* h, const double* params, double* Q, double dt, int nsteps) {
  Mesh* m = static_cast<Mesh*>(h);
  std::string err;
  return step(*m, read_params(params), Q, dt, nsteps, err);
}

// Implicit backward-Euler steps with kmax Jacobi iterations (Section 4).
int oracle_step_implicit(void* h, const double* params, double* Q, double dt, int nsteps,
                         int kmax) {
  Mesh* m = static_cast<Mesh*>(h);
  std::string err;
  return step_implicit(*m, read_params(params), Q, dt, nsteps, kmax, err);
}

// S2O4 with a forward tangent: Q and dQ are advanced together.
int oracle_step_jvp(void* h, const double* params, double* Q, double* dQ, double dt, int nsteps) {
  Mesh* m = static_cast<Mesh*>(h);
  const size_t len = 5 * (size_t)m->n_cells;
  std::vector<Dual> q(len);
  for (size_t k = 0; k < len; ++k) q[k] = Dual(Q[k], dQ[k]);
  std::string err;
  const int st = step(*m, read_params(params), q.data(), dt, nsteps, err);
  for (size_t k = 0; k < len; ++k) {
    Q[k] = q[k].v;
    dQ[k] = q[k].d;
  }
  return st;
}

void oracle_s2o4_stage1(int64_t len, const double* Q, const double* L, const double* Lt,
                        double dt, double* Qs) {
  s2o4_stage1((size_t)len, Q, L, Lt, dt, Qs);
}
void oracle_s2o4_stage2(int64_t len, const double* Q, const double* L, const double* Lt,
                        const double* Lts, double dt, double* Qn) {
  s2o4_stage2((size_t)len, Q, L, Lt, Lts, dt, Qn);
}

// Time step: dt = cfl * min_i h_i / (|U_i| + c_i + 2 nu_i / h_i), h_i = |Omega_i| / max face area.
int oracle_max_dt(void* h, const double* params, const double* Q, double cfl, double* dt) {
  Mesh* m = static_cast<Mesh*>(h);
  const Params P = read_params(params);
  const int n = m->n_cells;
  double best = 1e300;
  for (int i = 0; i < n; ++i) {
    const Cell& c = m->cells[i];
    double amax = 0;
    for (int f : c.face_id) amax = std::max(amax, m->faces[f].area);
    const double hi = c.vol / amax;
    double q[5];
    for (int v = 0; v < 5; ++v) q[v] = Q[v * (size_t)n + i];
    Prim<double> w;
    if (!primitive(q, P.gamma, w)) return ST_NONPHYS;
    const double speed = std::sqrt(w.U * w.U + w.V * w.V + w.W * w.W);
    const double cs = std::sqrt(P.gamma * w.p / w.rho);
    const double nu = viscosity(P, w.p / w.rho) / w.rho;
    best = std::min(best, hi / (speed + cs + 2.0 * nu / hi));
  }
  *dt = cfl * best;
  return ST_OK;
}

}  // extern "C"

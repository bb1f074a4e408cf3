// FP64 geometry precompute on the device: cell quadrature (27-point Gauss on the trilinear map,
// Section 2), face Gauss data (2x2 Gauss on the bilinear map, Eq. flux-qud), and the
// least-squares pseudo-inverses of the big stencils and sub-stencils (Section 2).
#include <cuda_runtime.h>

#include <cmath>

#include "gks_device.cuh"

namespace gks {
namespace {

constexpr int kThreads = 128;

__device__ __forceinline__ void set_flag(int* flag, int bit) { atomicOr(flag, bit); }

// 3-point Gauss-Legendre on [-1/2, 1/2].
__device__ __forceinline__ double g3x(int i) {
  return i == 0 ? -0.3872983346207417 : (i == 1 ? 0.0 : 0.3872983346207417);
}
__device__ __forceinline__ double g3w(int i) { return i == 1 ? 4.0 / 9.0 : 5.0 / 18.0; }

// Per cell: volume, centroid, |Omega|^(1/3), scaled second central moments; flags a cell whose
// trilinear Jacobian is not positive at every quadrature point.
__global__ void k_geom_cells(int64_t nc, const double* __restrict__ cell_x, double* vol,
                             double* ivol, double* cen, double* hh, double* mom, int* flag) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nc) return;
  double X[8][3];
  double o[3] = {0, 0, 0};
  for (int s = 0; s < 8; ++s)
    for (int a = 0; a < 3; ++a) {
      X[s][a] = cell_x[24 * i + 3 * s + a];
      o[a] += 0.125 * X[s][a];
    }
  // slot s sits at corner (sx, sy, sz) of [-1/2,1/2]^3 with this sign pattern
  const int sx[8] = {-1, 1, 1, -1, -1, 1, 1, -1};
  const int sy[8] = {-1, -1, 1, 1, -1, -1, 1, 1};
  const int sz[8] = {-1, -1, -1, -1, 1, 1, 1, 1};
  double m0 = 0, m1[3] = {0, 0, 0}, m2[6] = {0, 0, 0, 0, 0, 0};
  bool ok = true;
  for (int p = 0; p < 3; ++p)
    for (int q = 0; q < 3; ++q)
      for (int r = 0; r < 3; ++r) {
        const double xi = g3x(p), et = g3x(q), ze = g3x(r);
        double x[3] = {0, 0, 0}, J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        for (int s = 0; s < 8; ++s) {
          const double fx = 0.5 + sx[s] * xi, fy = 0.5 + sy[s] * et, fz = 0.5 + sz[s] * ze;
          const double w = fx * fy * fz;
          const double dx = sx[s] * fy * fz, dy = fx * sy[s] * fz, dz = fx * fy * sz[s];
          for (int a = 0; a < 3; ++a) {
            const double xs = X[s][a] - o[a];
            x[a] += xs * w;
            J[a][0] += xs * dx;
            J[a][1] += xs * dy;
            J[a][2] += xs * dz;
          }
        }
        const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                           J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                           J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
        if (!(det > 0.0)) ok = false;
        const double wt = g3w(p) * g3w(q) * g3w(r) * det;
        m0 += wt;
        for (int a = 0; a < 3; ++a) m1[a] += wt * x[a];
        m2[0] += wt * x[0] * x[0];
        m2[1] += wt * x[1] * x[1];
        m2[2] += wt * x[2] * x[2];
        m2[3] += wt * x[0] * x[1];
        m2[4] += wt * x[0] * x[2];
        m2[5] += wt * x[1] * x[2];
      }
  if (!ok) set_flag(flag, kErrInverted);
  const double c[3] = {m1[0] / m0, m1[1] / m0, m1[2] / m0};
  const double h = cbrt(m0);
  vol[i] = m0;
  ivol[i] = 1.0 / m0;
  hh[i] = h;
  for (int a = 0; a < 3; ++a) cen[3 * i + a] = o[a] + c[a];
  // central moments from raw moments about the vertex mean
  const int pa[6] = {0, 1, 2, 0, 0, 1}, pb[6] = {0, 1, 2, 1, 2, 2};
  for (int k = 0; k < 6; ++k) mom[k * nc + i] = (m2[k] / m0 - c[pa[k]] * c[pb[k]]) / (h * h);
}

// Per face: Gauss points, unit normals, area weights; offsets of each point from the owner's
// centroid and from the neighbour's centroid carried into the owner frame.
template <class R>
__global__ void k_geom_faces(int64_t nf, const double* __restrict__ f_vert,
                             const double* __restrict__ f_shift, const int32_t* __restrict__ f_owner,
                             const int32_t* __restrict__ f_nb, const double* __restrict__ cen,
                             double* farea, R* fgp) {
  const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= nf) return;
  double V[4][3];
  for (int k = 0; k < 4; ++k)
    for (int a = 0; a < 3; ++a) V[k][a] = f_vert[12 * f + 3 * k + a];
  const int32_t o = f_owner[f], nb = f_nb[f];
  double co[3], cn[3];
  for (int a = 0; a < 3; ++a) {
    co[a] = cen[3 * o + a];
    cn[a] = nb >= 0 ? cen[3 * nb + a] + f_shift[3 * f + a] : co[a];
  }
  // slots: v0 (-,-) v1 (-,+) v2 (+,+) v3 (+,-) in (eta, zeta)
  const double se[4] = {-1, -1, 1, 1}, sz[4] = {-1, 1, 1, -1};
  const double gp = 0.28867513459481287;  // sqrt(3)/6
  const int64_t stride = 4 * nf;
  double area = 0;
  for (int g = 0; g < 4; ++g) {
    const double eta = (g & 2) ? gp : -gp, zeta = (g & 1) ? gp : -gp;
    double x[3] = {0, 0, 0}, xe[3] = {0, 0, 0}, xz[3] = {0, 0, 0};
    for (int k = 0; k < 4; ++k) {
      const double fe = 0.5 + se[k] * eta, fz = 0.5 + sz[k] * zeta;
      for (int a = 0; a < 3; ++a) {
        x[a] += V[k][a] * fe * fz;
        xe[a] += V[k][a] * se[k] * fz;
        xz[a] += V[k][a] * fe * sz[k];
      }
    }
    const double n[3] = {xe[1] * xz[2] - xe[2] * xz[1], xe[2] * xz[0] - xe[0] * xz[2],
                         xe[0] * xz[1] - xe[1] * xz[0]};
    const double len = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    const int64_t idx = 4 * f + g;
    for (int a = 0; a < 3; ++a) {
      fgp[a * stride + idx] = (R)(x[a] - co[a]);
      fgp[(3 + a) * stride + idx] = (R)(x[a] - cn[a]);
      fgp[(6 + a) * stride + idx] = (R)(n[a] / len);
    }
    fgp[9 * stride + idx] = (R)(0.25 * len);
    area += 0.25 * len;
  }
  farea[f] = area;
}

// Per cell: |Omega| / (largest face area), the length used by the time-step bound.
__global__ void k_geom_hdt(int64_t nc, const int32_t* __restrict__ cf_ptr,
                           const int32_t* __restrict__ cf_idx, const double* __restrict__ farea,
                           const double* __restrict__ vol, double* hdt) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nc) return;
  double amax = 0;
  for (int k = cf_ptr[i]; k < cf_ptr[i + 1]; ++k) amax = fmax(amax, farea[cf_idx[k] >> 1]);
  hdt[i] = vol[i] / amax;
}

// Householder QR of the m x n matrix A (column-major, lda = m) in place; beta and rdiag of
// length n. Returns false when a diagonal of R is negligible (rank deficient).
__device__ bool qr_inplace(double* A, int m, int n, double* beta, double* rdiag) {
  double scale = 0;
  for (int k = 0; k < m * n; ++k) scale = fmax(scale, fabs(A[k]));
  for (int j = 0; j < n; ++j) {
    double s = 0;
    for (int i = j; i < m; ++i) s += A[i + j * m] * A[i + j * m];
    const double nrm = sqrt(s);
    if (!(nrm > 1e-12 * scale)) return false;
    const double alpha = A[j + j * m] > 0 ? -nrm : nrm;
    A[j + j * m] -= alpha;
    double vv = 0;
    for (int i = j; i < m; ++i) vv += A[i + j * m] * A[i + j * m];
    beta[j] = 2.0 / vv;
    for (int c = j + 1; c < n; ++c) {
      double d = 0;
      for (int i = j; i < m; ++i) d += A[i + j * m] * A[i + c * m];
      d *= beta[j];
      for (int i = j; i < m; ++i) A[i + c * m] -= d * A[i + j * m];
    }
    rdiag[j] = alpha;
  }
  return true;
}

// Column k of the pseudo-inverse R^{-1} Q^T of a factored matrix, written to out[0..n).
__device__ void pinv_column(const double* A, int m, int n, const double* beta, const double* rdiag,
                            int k, double* x, double* out) {
  for (int i = 0; i < m; ++i) x[i] = (i == k) ? 1.0 : 0.0;
  for (int j = 0; j < n; ++j) {
    double d = 0;
    for (int i = j; i < m; ++i) d += A[i + j * m] * x[i];
    d *= beta[j];
    for (int i = j; i < m; ++i) x[i] -= d * A[i + j * m];
  }
  for (int j = n - 1; j >= 0; --j) {
    double s = x[j];
    for (int c = j + 1; c < n; ++c) s -= A[j + c * m] * out[c];
    out[j] = s / rdiag[j];
  }
}

// Per cell: rows of the big-stencil system (mean of each scaled monomial over the member cell,
// minus its mean over the target cell), computed from member centroids and second moments
// (exact for the quadratic basis); QR-based pseudo-inverses of the big stencil (9 x K) and of
// every sub-stencil (3 x k_m).
template <class R>
__global__ void __launch_bounds__(kThreads) k_geom_ls(
    int64_t nc, const int32_t* __restrict__ st_ptr, const int32_t* __restrict__ st_idx,
    const double* __restrict__ st_xf, const uint8_t* __restrict__ st_sub,
    const int8_t* __restrict__ n_sub, const int32_t* __restrict__ t_st,
    const int32_t* __restrict__ t_sb, const uint64_t* __restrict__ t_cnt,
    const double* __restrict__ cen, const double* __restrict__ hh, const double* __restrict__ mom,
    R* Ap, R* Bp, int* flag, int* bad_cell) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nc) return;
  const int s0 = st_ptr[i], K = st_ptr[i + 1] - s0;
  if (K > kMaxStencil || K < 9) {
    atomicOr(flag, kErrSingular);
    atomicMin(bad_cell, (int)i);
    return;
  }
  double A[kMaxStencil * 9];
  double beta[9], rd[9], x[kMaxStencil], col[9];
  const double h0 = hh[i];
  const double c0[3] = {cen[3 * i], cen[3 * i + 1], cen[3 * i + 2]};
  double m0[6];
  for (int k = 0; k < 6; ++k) m0[k] = mom[k * nc + i];
  const int pa[6] = {0, 1, 2, 0, 0, 1}, pb[6] = {0, 1, 2, 1, 2, 2};
  for (int k = 0; k < K; ++k) {
    const int j = st_idx[s0 + k] & kCellMask;
    const double* xf = st_xf + 6 * (int64_t)(s0 + k);
    double d[3];
    for (int a = 0; a < 3; ++a) d[a] = (xf[a] * cen[3 * j + a] + xf[3 + a] - c0[a]) / h0;
    const double hj = hh[j], r2 = (hj * hj) / (h0 * h0);
    for (int a = 0; a < 3; ++a) A[k + a * K] = d[a];
    for (int q = 0; q < 6; ++q) {
      const double mj = mom[q * nc + j] * xf[pa[q]] * xf[pb[q]];
      A[k + (3 + q) * K] = d[pa[q]] * d[pb[q]] + mj * r2 - m0[q];
    }
  }
  // sub-stencils first (they only need the linear columns); entries sub-stencil major, per tile
  // slot one record of four values per lane (the three pseudo-inverse coefficients and the
  // member index: [slot][lane][4], one 16-byte load on the FP32 path)
  const int M = n_sub[i];
  const int64_t tile = i / kTile;
  const int lane = (int)(i % kTile);
  const uint64_t tc = t_cnt[tile];
  int slot0 = 0;  // first slot of sub-stencil s within the tile
  for (int s = 0; s < M; ++s) {
    double S[kMaxStencil * 3];
    int idx[kMaxStencil];
    int km = 0;
    for (int k = 0; k < K; ++k)
      if (st_sub[s0 + k] >> s & 1) idx[km++] = k;
    for (int r = 0; r < km; ++r)
      for (int a = 0; a < 3; ++a) S[r + a * km] = A[idx[r] + a * K];
    double sb[3], srd[3];
    if (km < 3 || !qr_inplace(S, km, 3, sb, srd)) {
      atomicOr(flag, kErrSingular);
      atomicMin(bad_cell, (int)i);
      return;
    }
    for (int r = 0; r < km; ++r) {
      double out[3];
      pinv_column(S, km, 3, sb, srd, r, x, out);
      const int64_t slot = (int64_t)t_sb[tile] + slot0 + r;
      R* rec = Bp + 4 * (slot * kTile + lane);
      for (int a = 0; a < 3; ++a) rec[a] = (R)out[a];
      rec[3] = (R)idx[r];  // member index, exact in either precision
    }
    slot0 += (int)((tc >> (8 * s)) & 0xffu);
  }
  if (!qr_inplace(A, K, 9, beta, rd)) {
    atomicOr(flag, kErrSingular);
    atomicMin(bad_cell, (int)i);
    return;
  }
  for (int k = 0; k < K; ++k) {
    pinv_column(A, K, 9, beta, rd, k, x, col);
    const int64_t row = (int64_t)t_st[tile] + k;
    for (int n = 0; n < 9; ++n) Ap[((9 * row) + n) * kTile + lane] = (R)col[n];
  }
}

template <class R>
__global__ void k_cast_cells(int64_t nc, const double* __restrict__ hh, const double* __restrict__ mom,
                             const double* __restrict__ ivol, R* h_out, R* mom_out, R* ivol_out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nc) return;
  h_out[i] = (R)hh[i];
  for (int k = 0; k < 6; ++k) mom_out[k * nc + i] = (R)mom[k * nc + i];
  if (sizeof(R) == 4) {  // float-float pair
    const float hi = (float)ivol[i];
    ivol_out[2 * i] = (R)hi;
    ivol_out[2 * i + 1] = (R)(ivol[i] - (double)hi);
  } else {
    ivol_out[i] = (R)ivol[i];
  }
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// The 27 Gauss points (3 per direction on [-1/2,1/2]^3 mapped by the trilinear map) and their
// weights times |J| for every cell, written at the caller's cell index.
__global__ void k_cell_quadrature(int64_t nc, const double* __restrict__ cell_x,
                                  const int32_t* __restrict__ perm, double* xq, double* wq) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nc) return;
  double X[8][3];
  for (int s = 0; s < 8; ++s)
    for (int a = 0; a < 3; ++a) X[s][a] = cell_x[24 * i + 3 * s + a];
  const int sx[8] = {-1, 1, 1, -1, -1, 1, 1, -1};
  const int sy[8] = {-1, -1, 1, 1, -1, -1, 1, 1};
  const int sz[8] = {-1, -1, -1, -1, 1, 1, 1, 1};
  const int64_t c = perm[i];
  int g = 0;
  for (int p = 0; p < 3; ++p)
    for (int q = 0; q < 3; ++q)
      for (int r = 0; r < 3; ++r, ++g) {
        const double xi = g3x(p), et = g3x(q), ze = g3x(r);
        double x[3] = {0, 0, 0}, J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        for (int s = 0; s < 8; ++s) {
          const double fx = 0.5 + sx[s] * xi, fy = 0.5 + sy[s] * et, fz = 0.5 + sz[s] * ze;
          for (int a = 0; a < 3; ++a) {
            x[a] += X[s][a] * fx * fy * fz;
            J[a][0] += X[s][a] * sx[s] * fy * fz;
            J[a][1] += X[s][a] * fx * sy[s] * fz;
            J[a][2] += X[s][a] * fx * fy * sz[s];
          }
        }
        const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                           J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                           J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
        for (int a = 0; a < 3; ++a) xq[(27 * c + g) * 3 + a] = x[a];
        wq[27 * c + g] = g3w(p) * g3w(q) * g3w(r) * det;
      }
}

}  // namespace

void launch_cell_quadrature(const DevMesh& m, double* xq, double* wq, cudaStream_t st) {
  k_cell_quadrature<<<blocks_for(m.nc, kThreads), kThreads, 0, st>>>(m.nc, m.cell_x, m.perm, xq, wq);
}

void launch_geom_cells(const DevMesh& m, const Geo64& g, int* flag, cudaStream_t st) {
  k_geom_cells<<<blocks_for(m.nc, kThreads), kThreads, 0, st>>>(m.nc, m.cell_x, g.vol, g.ivol, g.cen, g.h,
                                                                g.mom, flag);
}
template <class R>
void launch_geom_faces(const DevMesh& m, const Geo64& g, GeoR<R>& gr, cudaStream_t st) {
  k_geom_faces<R><<<blocks_for(m.nf, kThreads), kThreads, 0, st>>>(
      m.nf, m.f_vert, m.f_shift, m.f_owner, m.f_nb, g.cen, g.farea, gr.fgp);
}
void launch_geom_hdt(const DevMesh& m, const Geo64& g, cudaStream_t st) {
  k_geom_hdt<<<blocks_for(m.nc, kThreads), kThreads, 0, st>>>(m.nc, m.cf_ptr, m.cf_idx, g.farea,
                                                              g.vol, g.hdt);
}
template <class R>
void launch_geom_ls(const DevMesh& m, const Geo64& g, GeoR<R>& gr, int* flag, int* bad_cell,
                    cudaStream_t st) {
  // padding of the tile layouts must read as zero coefficients
  cudaMemsetAsync(gr.Ap, 0, sizeof(R) * 9 * kTile * (size_t)m.n_tslots, st);
  cudaMemsetAsync(gr.Bp, 0, sizeof(R) * 4 * kTile * (size_t)m.n_tsb, st);
  k_geom_ls<R><<<blocks_for(m.nc, 64), 64, 0, st>>>(m.nc, m.st_ptr, m.st_idx, m.st_xf, m.st_sub,
                                                      m.n_sub, m.t_st, m.t_sb, m.t_cnt, g.cen, g.h,
                                                      g.mom, gr.Ap, gr.Bp, flag, bad_cell);
}
template <class R>
void launch_cast_cells(const DevMesh& m, const Geo64& g, GeoR<R>& gr, cudaStream_t st) {
  k_cast_cells<R><<<blocks_for(m.nc, kThreads), kThreads, 0, st>>>(m.nc, g.h, g.mom, g.ivol, gr.h,
                                                                  gr.mom, gr.ivol);
}

// Unit normal (out of the owner) and area of every face, [nf][4] = (n, S), from its area vector
// int X_eta x X_zeta over [-1/2,1/2]^2 = 1/2 (v4 - v2) x (v3 - v1) for the cyclic vertex list
// v1..v4 (exact for the bilinear face: the integrand is bilinear, its mean is its centre value).
template <class R>
__global__ void k_face_normals(int64_t nf, const double* __restrict__ f_vert, R* out) {
  const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= nf) return;
  const double* v = f_vert + 12 * f;
  double a[3], b[3];
  for (int c = 0; c < 3; ++c) {
    a[c] = v[9 + c] - v[3 + c];  // v4 - v2
    b[c] = v[6 + c] - v[c];      // v3 - v1
  }
  const double S[3] = {0.5 * (a[1] * b[2] - a[2] * b[1]), 0.5 * (a[2] * b[0] - a[0] * b[2]),
                       0.5 * (a[0] * b[1] - a[1] * b[0])};
  const double area = sqrt(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
  for (int c = 0; c < 3; ++c) out[4 * f + c] = (R)(S[c] / area);
  out[4 * f + 3] = (R)area;
}
template <class R>
void launch_face_normals(const DevMesh& m, R* out, cudaStream_t st) {
  k_face_normals<R><<<blocks_for(m.nf, kThreads), kThreads, 0, st>>>(m.nf, m.f_vert, out);
}
template void launch_face_normals<double>(const DevMesh&, double*, cudaStream_t);
template void launch_face_normals<float>(const DevMesh&, float*, cudaStream_t);

template void launch_geom_faces<double>(const DevMesh&, const Geo64&, GeoR<double>&, cudaStream_t);
template void launch_geom_faces<float>(const DevMesh&, const Geo64&, GeoR<float>&, cudaStream_t);
template void launch_geom_ls<double>(const DevMesh&, const Geo64&, GeoR<double>&, int*, int*,
                                     cudaStream_t);
template void launch_geom_ls<float>(const DevMesh&, const Geo64&, GeoR<float>&, int*, int*,
                                    cudaStream_t);
template void launch_cast_cells<double>(const DevMesh&, const Geo64&, GeoR<double>&, cudaStream_t);
template void launch_cast_cells<float>(const DevMesh&, const Geo64&, GeoR<float>&, cudaStream_t);

}  // namespace gks

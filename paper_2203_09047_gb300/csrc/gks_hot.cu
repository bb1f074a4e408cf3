// Hot-path kernels: WENO reconstruction per cell (Section 2), gas-kinetic flux per face Gauss
// point (Section 3.2), per-cell gather of face fluxes with the two-stage fourth-order update
// (Section 3.3), the time-step bound, and caller-order permutations.
#include <cuda_runtime.h>

#include <cfloat>
#include <cmath>

#include "gks_device.cuh"
#include "gks_kinetic.cuh"

namespace gks {
namespace {

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// ------------------------------------------------------------------------------------------
// Reconstruction: one thread per cell, one pass per conserved variable. For variable v:
//   dq_k = Q_k - Q_0 over the big stencil (formed in FP64, mirrored momentum sign-flipped),
//   a    = A+ dq            (quadratic P0, 9 coefficients in centred scaled coordinates)
//   b_m  = B_m dq|S_m       (linear P_m, 3 coefficients each)
//   beta_0, beta_m (Eq. indicator), tau, omega, omega-bar (Section 2),
//   C    = (wb_0/g_0) a + sum_m (wb_m - wb_0 g_m/g_0) b_m    (Eq. weno as one polynomial),
// written as 10 coefficients of the polynomial in physical offsets from the centroid.
template <class R>
__global__ void __launch_bounds__(128) k_recon(
    int64_t nc, const double* __restrict__ Q, const int32_t* __restrict__ st_ptr,
    const int32_t* __restrict__ st_idx, const uint8_t* __restrict__ st_sub,
    const int8_t* __restrict__ n_sub, const int32_t* __restrict__ sb_ptr,
    const R* __restrict__ Ap, const R* __restrict__ Bp, const R* __restrict__ mom,
    const R* __restrict__ hcell, R wg, R weps, int wpow, R* __restrict__ poly) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nc) return;
  const int s0 = st_ptr[i];
  const int K = st_ptr[i + 1] - s0;
  const int M = n_sub[i];
  const R* A = Ap + 9 * (int64_t)s0;
  const R* B = Bp + 3 * (int64_t)sb_ptr[i];
  R m2[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) m2[q] = mom[q * nc + i];
  const R h = hcell[i];
  const R ih = R(1) / h, ih2 = ih * ih;
  const R g0 = R(1) - wg * R(M);
  for (int v = 0; v < 5; ++v) {
    const double q0 = Q[v * nc + i];
    R a[9], b[kMaxSub][3];
#pragma unroll
    for (int n = 0; n < 9; ++n) a[n] = R(0);
#pragma unroll
    for (int s = 0; s < kMaxSub; ++s) b[s][0] = b[s][1] = b[s][2] = R(0);
    int bp = 0;
    for (int k = 0; k < K; ++k) {
      const int32_t e = st_idx[s0 + k];
      double qk = Q[v * nc + (e & kCellMask)];
      if (v >= 1 && v <= 3 && ((e >> (kFlipShift + v - 1)) & 1)) qk = -qk;
      const R d = (R)(qk - q0);
#pragma unroll
      for (int n = 0; n < 9; ++n) a[n] += A[n * K + k] * d;
      const unsigned sm = st_sub[s0 + k];
#pragma unroll
      for (int s = 0; s < kMaxSub; ++s) {
        if (sm >> s & 1u) {
          b[s][0] += B[bp] * d;
          b[s][1] += B[bp + 1] * d;
          b[s][2] += B[bp + 2] * d;
          bp += 3;
        }
      }
    }
    // smoothness indicators in scaled coordinates: |l|=1 terms are cell means of the squared
    // first derivatives (linear in y), |l|=2 terms are the squared second derivatives
    const R gx[3] = {R(2) * a[3], a[6], a[7]};
    const R gy[3] = {a[6], R(2) * a[4], a[8]};
    const R gz[3] = {a[7], a[8], R(2) * a[5]};
    auto qform = [&](const R g[3]) {
      return m2[0] * g[0] * g[0] + m2[1] * g[1] * g[1] + m2[2] * g[2] * g[2] +
             R(2) * (m2[3] * g[0] * g[1] + m2[4] * g[0] * g[2] + m2[5] * g[1] * g[2]);
    };
    const R beta0 = a[0] * a[0] + a[1] * a[1] + a[2] * a[2] + qform(gx) + qform(gy) + qform(gz) +
                    R(4) * (a[3] * a[3] + a[4] * a[4] + a[5] * a[5]) + a[6] * a[6] + a[7] * a[7] +
                    a[8] * a[8];
    R beta[kMaxSub];
    R tau = R(0);
#pragma unroll
    for (int s = 0; s < kMaxSub; ++s) {
      beta[s] = b[s][0] * b[s][0] + b[s][1] * b[s][1] + b[s][2] * b[s][2];
      if (s < M) tau += fabs(beta0 - beta[s]);
    }
    tau /= R(M);
    auto weight = [&](R gam, R bet) {
      const R r = tau / (bet + weps);
      R p = r;
      for (int e = 1; e < wpow; ++e) p *= r;
      return gam * (R(1) + p);
    };
    const R w0 = weight(g0, beta0);
    R w[kMaxSub];
    R sum = w0;
#pragma unroll
    for (int s = 0; s < kMaxSub; ++s) {
      w[s] = s < M ? weight(wg, beta[s]) : R(0);
      sum += w[s];
    }
    const R is = R(1) / sum;
    const R wb0 = w0 * is;
    const R c_a = wb0 / g0;
    R C[9];
#pragma unroll
    for (int n = 0; n < 9; ++n) C[n] = c_a * a[n];
#pragma unroll
    for (int s = 0; s < kMaxSub; ++s) {
      if (s < M) {
        const R cs = w[s] * is - wb0 * wg / g0;
        C[0] += cs * b[s][0];
        C[1] += cs * b[s][1];
        C[2] += cs * b[s][2];
      }
    }
    // polynomial in physical offsets d = x - centroid:
    //   Q = c0 + c1 dx + c2 dy + c3 dz + c4 dx^2 + c5 dy^2 + c6 dz^2 + c7 dxdy + c8 dxdz + c9 dydz
    const R c0 = (R)q0 - (C[3] * m2[0] + C[4] * m2[1] + C[5] * m2[2] + C[6] * m2[3] +
                          C[7] * m2[4] + C[8] * m2[5]);
    R* out = poly + (int64_t)(10 * v) * nc + i;
    out[0] = c0;
    out[1 * nc] = C[0] * ih;
    out[2 * nc] = C[1] * ih;
    out[3 * nc] = C[2] * ih;
#pragma unroll
    for (int n = 3; n < 9; ++n) out[(n + 1) * nc] = C[n] * ih2;
  }
}

// Coefficient accessor of one cell's polynomial in the SoA array [50][nc].
template <class R>
struct PolyRef {
  const R* __restrict__ p;
  int64_t nc, c;
  __device__ __forceinline__ R operator()(int v, int j) const { return p[(int64_t)(10 * v + j) * nc + c]; }
};

// ------------------------------------------------------------------------------------------
// Flux: four consecutive threads per face, one per Gauss point. Each evaluates both sides'
// reconstructions, rotates into the local frame (n1 normal, n2 = n1 x e_k normalised with e_k
// the axis least aligned with n1, n3 = n1 x n2), computes F^n and dF/dt, rotates back and
// weights by the quadrature weight; the four are summed with shuffles and written once.
template <class R>
__global__ void __launch_bounds__(128) k_flux(
    int64_t nf, int64_t nc, const int32_t* __restrict__ f_owner, const int32_t* __restrict__ f_nb,
    const int8_t* __restrict__ f_wall, const R* __restrict__ fgp, const R* __restrict__ poly,
    FluxParams<R> P, R dt, R* __restrict__ fface, int* flag) {
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t f = gid >> 2;
  const bool active = f < nf;
  R acc[10];
#pragma unroll
  for (int q = 0; q < 10; ++q) acc[q] = R(0);
  int wall = -1;
  if (active) {
    const int64_t stride = 4 * nf;
    const int32_t o = f_owner[f], nb = f_nb[f];
    wall = f_wall[f];
    R dl[3], dr[3], n1[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      dl[a] = fgp[a * stride + gid];
      dr[a] = fgp[(3 + a) * stride + gid];
      n1[a] = fgp[(6 + a) * stride + gid];
    }
    const R w = fgp[9 * stride + gid];
    R vl[5], gl[5][3], vr[5], gr[5][3];
    eval_poly(PolyRef<R>{poly, nc, o}, dl, vl, gl);
    if (nb >= 0) {
      eval_poly(PolyRef<R>{poly, nc, nb}, dr, vr, gr);
    } else {
      // mirror image of the owner across the wall plane (axis `wall`)
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const R sv = (v == 1 + wall) ? R(-1) : R(1);
        vr[v] = sv * vl[v];
#pragma unroll
        for (int a = 0; a < 3; ++a) gr[v][a] = (a == wall ? -sv : sv) * gl[v][a];
      }
    }
    if (!gp_flux_global(P, vl, gl, vr, gr, n1, w, dt, acc)) atomicOr(flag, kErrNonphysical);
  }
  // sum the four Gauss points of the face (lanes 4f .. 4f+3 of one warp)
#pragma unroll
  for (int q = 0; q < 10; ++q) {
    acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], 1);
    acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], 2);
  }
  if (active && (gid & 3) == 0) {
    if (wall >= 0) {
      // reflecting wall: only the normal momentum component survives
#pragma unroll
      for (int v = 0; v < 5; ++v)
        if (v != 1 + wall) acc[v] = acc[5 + v] = R(0);
    }
#pragma unroll
    for (int q = 0; q < 10; ++q) fface[q * nf + f] = acc[q];
  }
}

template <class R>
__device__ __forceinline__ bool physical(const double q[5], double gamma) {
  const double ke = 0.5 * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]) / q[0];
  const double p = (gamma - 1.0) * (q[4] - ke);
  return q[0] > 0.0 && p > 0.0;
}

// Per cell: L = -(1/|Omega|) sum_f s_f F_f in the cell's fixed face order (FP64), then the
// requested update.
template <class R>
__global__ void __launch_bounds__(256) k_gather(
    int64_t nc, int64_t nf, const int32_t* __restrict__ cf_ptr, const int32_t* __restrict__ cf_idx,
    const R* __restrict__ fface, const double* __restrict__ vol, int mode, double dt, double gamma,
    double* __restrict__ L, double* __restrict__ Lt, double* __restrict__ Qn,
    double* __restrict__ Qs, int* flag) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nc) return;
  double s[10];
#pragma unroll
  for (int q = 0; q < 10; ++q) s[q] = 0.0;
  for (int k = cf_ptr[i]; k < cf_ptr[i + 1]; ++k) {
    const int32_t e = cf_idx[k];
    const int64_t f = e >> 1;
    const double sg = (e & 1) ? 1.0 : -1.0;  // owner loses the outward flux
#pragma unroll
    for (int q = 0; q < 10; ++q) s[q] += sg * (double)fface[q * nf + f];
  }
  const double iv = 1.0 / vol[i];
  double l[5], lt[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    l[v] = s[v] * iv;
    lt[v] = s[5 + v] * iv;
  }
  if (mode == 0) {
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      L[v * nc + i] = l[v];
      Lt[v * nc + i] = lt[v];
    }
    return;
  }
  double q[5];
  if (mode == 1) {
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      L[v * nc + i] = l[v];
      Lt[v * nc + i] = lt[v];
      q[v] = Qn[v * nc + i] + 0.5 * dt * l[v] + (dt * dt / 8.0) * lt[v];
      Qs[v * nc + i] = q[v];
    }
  } else {
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      q[v] = Qn[v * nc + i] + dt * L[v * nc + i] +
             (dt * dt / 6.0) * (Lt[v * nc + i] + 2.0 * lt[v]);
      Qn[v * nc + i] = q[v];
    }
  }
  if (!physical<R>(q, gamma)) atomicOr(flag, kErrNonphysical);
}

__global__ void k_permute_in(int64_t nc, const int32_t* __restrict__ perm,
                             const double* __restrict__ src, double* __restrict__ dst) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nc) return;
  const int64_t c = perm[i];
#pragma unroll
  for (int v = 0; v < 5; ++v) dst[v * nc + i] = src[v * nc + c];
}
__global__ void k_permute_out(int64_t nc, const int32_t* __restrict__ perm,
                              const double* __restrict__ src, double* __restrict__ dst) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nc) return;
  const int64_t c = perm[i];
#pragma unroll
  for (int v = 0; v < 5; ++v) dst[v * nc + c] = src[v * nc + i];
}
__global__ void k_check_state(int64_t nc, const double* __restrict__ Q, double gamma, int* flag) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nc) return;
  double q[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) q[v] = Q[v * nc + i];
  if (!physical<double>(q, gamma)) atomicOr(flag, kErrNonphysical);
}

constexpr int kDtThreads = 256;
constexpr int kDtMaxBlocks = 1024;

__global__ void __launch_bounds__(kDtThreads) k_dt_partial(int64_t nc, const double* __restrict__ Q,
                                                           const double* __restrict__ hdt,
                                                           double gamma, double mu,
                                                           double* partial) {
  __shared__ double red[kDtThreads / 32];
  double best = DBL_MAX;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nc;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double r = Q[i], mx = Q[nc + i], my = Q[2 * nc + i], mz = Q[3 * nc + i], E = Q[4 * nc + i];
    const double u2 = (mx * mx + my * my + mz * mz) / (r * r);
    const double p = (gamma - 1.0) * (E - 0.5 * r * u2);
    const double c = sqrt(gamma * p / r);
    const double h = hdt[i];
    const double bound = h / (sqrt(u2) + c + 2.0 * mu / (r * h));
    best = fmin(best, bound);  // NaN states are caught by the state checks
  }
  for (int o = 16; o > 0; o >>= 1) best = fmin(best, __shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x < 32) {
    best = threadIdx.x < kDtThreads / 32 ? red[threadIdx.x] : DBL_MAX;
    for (int o = 16; o > 0; o >>= 1) best = fmin(best, __shfl_xor_sync(0xffffffffu, best, o));
    if (threadIdx.x == 0) partial[blockIdx.x] = best;
  }
}
__global__ void k_dt_final(const double* partial, int n, double* out) {
  __shared__ double red[32];
  double best = DBL_MAX;
  for (int k = threadIdx.x; k < n; k += blockDim.x) best = fmin(best, partial[k]);
  for (int o = 16; o > 0; o >>= 1) best = fmin(best, __shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x < 32) {
    best = threadIdx.x < (int)(blockDim.x / 32) ? red[threadIdx.x] : DBL_MAX;
    for (int o = 16; o > 0; o >>= 1) best = fmin(best, __shfl_xor_sync(0xffffffffu, best, o));
    if (threadIdx.x == 0) *out = best;
  }
}

}  // namespace

template <class R>
void launch_recon(const DevMesh& m, const GeoR<R>& g, const KParams<R>& p, const double* Q,
                  R* poly, cudaStream_t st) {
  k_recon<R><<<blocks_for(m.nc, 128), 128, 0, st>>>(m.nc, Q, m.st_ptr, m.st_idx, m.st_sub,
                                                      m.n_sub, m.sb_ptr, g.Ap, g.Bp, g.mom, g.h,
                                                      p.weno_gamma, p.weno_eps, p.weno_pow, poly);
}
template <class R>
void launch_flux(const DevMesh& m, const GeoR<R>& g, const KParams<R>& p, const R* poly,
                 double dt, R* fface, int* flag, cudaStream_t st) {
  FluxParams<R> fp;
  fp.gamma = p.gamma;
  fp.K = p.K;
  fp.mu = p.mu;
  fp.tau_eps = p.tau_eps;
  fp.tau_C = p.tau_C;
  fp.full = p.flux_mode;
  fp.tau_model = p.tau_model;
  k_flux<R><<<blocks_for(4 * m.nf, 128), 128, 0, st>>>(m.nf, m.nc, m.f_owner, m.f_nb, m.f_wall,
                                                         g.fgp, poly, fp, (R)dt, fface, flag);
}
template <class R>
void launch_gather(const DevMesh& m, const Geo64& g, const R* fface, int mode, double dt,
                   double gamma, double* L, double* Lt, double* Qn, double* Qs, int* flag,
                   cudaStream_t st) {
  k_gather<R><<<blocks_for(m.nc, 256), 256, 0, st>>>(m.nc, m.nf, m.cf_ptr, m.cf_idx, fface, g.vol,
                                                       mode, dt, gamma, L, Lt, Qn, Qs, flag);
}
void launch_permute_in(int64_t nc, const int32_t* perm, const double* src, double* dst,
                       cudaStream_t st) {
  k_permute_in<<<blocks_for(nc, 256), 256, 0, st>>>(nc, perm, src, dst);
}
void launch_permute_out(int64_t nc, const int32_t* perm, const double* src, double* dst,
                        cudaStream_t st) {
  k_permute_out<<<blocks_for(nc, 256), 256, 0, st>>>(nc, perm, src, dst);
}
void launch_check_state(int64_t nc, const double* Q, double gamma, int* flag, cudaStream_t st) {
  k_check_state<<<blocks_for(nc, 256), 256, 0, st>>>(nc, Q, gamma, flag);
}
int dt_blocks(int64_t nc) {
  const int64_t b = (nc + kDtThreads - 1) / kDtThreads;
  return (int)(b < kDtMaxBlocks ? b : kDtMaxBlocks);
}
void launch_dt(int64_t nc, const double* Q, const double* hdt, double gamma, double mu,
               double* partial, int nblocks, double* out, cudaStream_t st) {
  k_dt_partial<<<nblocks, kDtThreads, 0, st>>>(nc, Q, hdt, gamma, mu, partial);
  k_dt_final<<<1, 256, 0, st>>>(partial, nblocks, out);
}

template void launch_recon<double>(const DevMesh&, const GeoR<double>&, const KParams<double>&,
                                   const double*, double*, cudaStream_t);
template void launch_recon<float>(const DevMesh&, const GeoR<float>&, const KParams<float>&,
                                  const double*, float*, cudaStream_t);
template void launch_flux<double>(const DevMesh&, const GeoR<double>&, const KParams<double>&,
                                  const double*, double, double*, int*, cudaStream_t);
template void launch_flux<float>(const DevMesh&, const GeoR<float>&, const KParams<float>&,
                                 const float*, double, float*, int*, cudaStream_t);
template void launch_gather<double>(const DevMesh&, const Geo64&, const double*, int, double, double,
                                    double*, double*, double*, double*, int*, cudaStream_t);
template void launch_gather<float>(const DevMesh&, const Geo64&, const float*, int, double, double,
                                   double*, double*, double*, double*, int*, cudaStream_t);

}  // namespace gks

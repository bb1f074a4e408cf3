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
// Gather copy of a state (48 bytes per cell, see Lay<R>) and the stencil differences taken
// from it. FP32 path: each value is kept as hi + lo floats, so Q_k - Q_0 is formed as
// (hi_k - hi_0) + (lo_k - lo_0) without FP64 arithmetic and is as accurate as rounding the
// FP64 difference to FP32. FP64 path: the FP64 values themselves.
template <class R>
struct Gq;
template <>
struct Gq<float> {
  float hi[5], lo[5];
  __device__ __forceinline__ void load(const float* __restrict__ QA, int64_t c) {
    const float4* p = reinterpret_cast<const float4*>(QA + 12 * c);
    const float4 a = __ldg(p), b = __ldg(p + 1), d = __ldg(p + 2);
    hi[0] = a.x; hi[1] = a.y; hi[2] = a.z; hi[3] = a.w; hi[4] = b.x;
    lo[0] = b.y; lo[1] = b.z; lo[2] = b.w; lo[3] = d.x; lo[4] = d.y;
  }
  __device__ __forceinline__ void flip(int v) { hi[v] = -hi[v]; lo[v] = -lo[v]; }
  __device__ __forceinline__ float minus(const Gq& c, int v) const {
    return (hi[v] - c.hi[v]) + (lo[v] - c.lo[v]);
  }
  __device__ __forceinline__ float value(int v) const { return hi[v] + lo[v]; }
  __device__ __forceinline__ float value_minus(int v, float x) const { return hi[v] + (lo[v] - x); }
  __device__ static void store(float* QA, int64_t c, const double q[5]) {
    float h[5], l[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      h[v] = (float)q[v];
      l[v] = (float)(q[v] - (double)h[v]);
    }
    float4* p = reinterpret_cast<float4*>(QA + 12 * c);
    p[0] = make_float4(h[0], h[1], h[2], h[3]);
    p[1] = make_float4(h[4], l[0], l[1], l[2]);
    p[2] = make_float4(l[3], l[4], 0.f, 0.f);
  }
};
template <>
struct Gq<double> {
  double q[5];
  __device__ __forceinline__ void load(const double* __restrict__ QA, int64_t c) {
    const double2* p = reinterpret_cast<const double2*>(QA + 6 * c);
    const double2 a = __ldg(p), b = __ldg(p + 1), d = __ldg(p + 2);
    q[0] = a.x; q[1] = a.y; q[2] = b.x; q[3] = b.y; q[4] = d.x;
  }
  __device__ __forceinline__ void flip(int v) { q[v] = -q[v]; }
  __device__ __forceinline__ double minus(const Gq& c, int v) const { return q[v] - c.q[v]; }
  __device__ __forceinline__ double value(int v) const { return q[v]; }
  __device__ __forceinline__ double value_minus(int v, double x) const { return q[v] - x; }
  __device__ static void store(double* QA, int64_t c, const double qq[5]) {
    double2* p = reinterpret_cast<double2*>(QA + 6 * c);
    p[0] = make_double2(qq[0], qq[1]);
    p[1] = make_double2(qq[2], qq[3]);
    p[2] = make_double2(qq[4], 0.0);
  }
};

// dq[v] = Q_member - Q_0 for one stencil entry (cell | mirrored-axis bits).
template <class R>
__device__ __forceinline__ void stencil_delta(const R* __restrict__ QA, int32_t e, const Gq<R>& c0,
                                              R dq[5]) {
  Gq<R> g;
  g.load(QA, e & kCellMask);
  const int fl = e >> kFlipShift;
  if (fl & 1) g.flip(1);
  if (fl & 2) g.flip(2);
  if (fl & 4) g.flip(3);
#pragma unroll
  for (int v = 0; v < 5; ++v) dq[v] = g.minus(c0, v);
}

// ------------------------------------------------------------------------------------------
// Reconstruction, one block of four warps per 32-cell tile (lane = cell). For each conserved
// variable v of each cell:
//   dq_k = Q_k - Q_0 over the big stencil                      (phase 1, all warps, to shared)
//   a    = A+ dq   (quadratic P0, 9 coefficients in centred scaled coordinates) and
//   b_m  = B_m dq|S_m (linear P_m) with beta_m (Eq. indicator); rows and sub-stencils are
//   spread over the four warps                                                       (phase 2)
//   beta_0, tau, omega, omega-bar (Section 2), one variable per warp               (phase 3)
//   C = (wb_0/g_0) a + sum_m (wb_m - wb_0 g_m/g_0) b_m, i.e. Eq. weno as one polynomial (phase 4)
// Output: 10 coefficients per variable of the polynomial in physical offsets from the centroid.
// Variables are split over the warps as warp w -> v = w, and warp 0 also takes v = 4.
constexpr int kReconWarps = 4;
constexpr int kReconThreads = kReconWarps * kTile;

template <class R>
struct ReconShared {
  R a[9][5][kTile];             // big-stencil coefficients
  R b[kMaxSub][3][5][kTile];    // sub-stencil coefficients
  R bet[kMaxSub][5][kTile];     // beta_m, then the sub-stencil factors of the combination
  R ca[5][kTile];               // factor of a in the combination
  // followed by dq[K][5][kTile]
};

template <class R>
__global__ void __launch_bounds__(kReconThreads) k_recon(
    int64_t nc, const R* __restrict__ QA, const int32_t* __restrict__ t_K,
    const uint64_t* __restrict__ t_cnt, const int32_t* __restrict__ t_st,
    const int32_t* __restrict__ t_sb, const int32_t* __restrict__ t_idx,
    const int8_t* __restrict__ n_sub, const R* __restrict__ Ap, const R* __restrict__ Bp,
    const R* __restrict__ mom, const R* __restrict__ hcell, R wg, R weps, int wpow,
    R* __restrict__ poly) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ReconShared<R>& sh = *reinterpret_cast<ReconShared<R>*>(smem_raw);
  R* sdq = reinterpret_cast<R*>(smem_raw + sizeof(ReconShared<R>));  // [k][v][lane]
  const int64_t tile = blockIdx.x;
  const int lane = threadIdx.x & (kTile - 1);
  const int warp = threadIdx.x / kTile;
  const int64_t i = tile * kTile + lane;
  const bool valid = i < nc;
  const int64_t ic = valid ? i : tile * kTile;  // padded lanes mirror the tile's first cell
  const int K = __ldg(t_K + tile);
  const uint64_t cnt = __ldg(t_cnt + tile);
  const int32_t* sidx = t_idx + (int64_t)__ldg(t_st + tile) * kTile + lane;
  const R* A = Ap + (int64_t)__ldg(t_st + tile) * 9 * kTile + lane;
  const R* Bt = Bp + (int64_t)__ldg(t_sb + tile) * 4 * kTile + lane;
  Gq<R> c0;
  c0.load(QA, ic);

  // phase 1: stencil differences, members split over the warps; the loops below are unrolled
  // so that several iterations' loads are in flight per warp
  for (int k0 = warp; k0 < K; k0 += 4 * kReconWarps) {
    // four members per batch: all index loads, then all state loads, then the differences
    int32_t e[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int k = k0 + u * kReconWarps;
      e[u] = k < K ? __ldg(sidx + k * kTile) : -1;
    }
    Gq<R> g[4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (e[u] >= 0) g[u].load(QA, e[u] & kCellMask);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (e[u] < 0) continue;
      const int fl = e[u] >> kFlipShift;
      if (fl & 1) g[u].flip(1);
      if (fl & 2) g[u].flip(2);
      if (fl & 4) g[u].flip(3);
      const int k = k0 + u * kReconWarps;
#pragma unroll
      for (int v = 0; v < 5; ++v) sdq[(5 * k + v) * kTile + lane] = g[u].minus(c0, v);
    }
  }
  __syncthreads();

  // phase 2, all warps: rows n = warp, warp + 4, warp + 8 of a = A+ dq, and the sub-stencil
  // fits b_m (m = warp, warp + 4) with their indicators beta_m = |b_m|^2 (scaled coordinates)
  for (int n = warp; n < 9; n += kReconWarps) {
    R acc[5] = {R(0), R(0), R(0), R(0), R(0)};
#pragma unroll 4
    for (int k = 0; k < K; ++k) {
      const R row = __ldg(A + (9 * k + n) * kTile);
#pragma unroll
      for (int v = 0; v < 5; ++v) acc[v] += row * sdq[(5 * k + v) * kTile + lane];
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) sh.a[n][v][lane] = acc[v];
  }
  {
    int slot = 0;
    for (int s = 0; s < warp; ++s) slot += (int)((cnt >> (8 * s)) & 0xffu);
    for (int s = warp; s < kMaxSub; s += kReconWarps) {
      const int cs = (int)((cnt >> (8 * s)) & 0xffu);
      const R* e = Bt + (int64_t)4 * kTile * slot;
      R b[3][5];
#pragma unroll
      for (int t = 0; t < 3; ++t)
#pragma unroll
        for (int v = 0; v < 5; ++v) b[t][v] = R(0);
#pragma unroll 2
      for (int j = 0; j < cs; ++j, e += 4 * kTile) {
        const int k = (int)__ldg(e + 3 * kTile);
        const R c[3] = {__ldg(e), __ldg(e + kTile), __ldg(e + 2 * kTile)};
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          const R dq = sdq[(5 * k + v) * kTile + lane];
#pragma unroll
          for (int t = 0; t < 3; ++t) b[t][v] += c[t] * dq;
        }
      }
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        sh.bet[s][v][lane] = b[0][v] * b[0][v] + b[1][v] * b[1][v] + b[2][v] * b[2][v];
#pragma unroll
        for (int t = 0; t < 3; ++t) sh.b[s][t][v][lane] = b[t][v];
      }
      // slots of the sub-stencils this warp skips (the other warps' ones)
      for (int q = s; q < s + kReconWarps && q < kMaxSub; ++q) slot += (int)((cnt >> (8 * q)) & 0xffu);
    }
  }
  __syncthreads();

  // phase 3: nonlinear weights, one variable per warp (warp 0 also does v = 4)
  const int M = n_sub[ic];
  const R g0 = R(1) - wg * R(M);
  R m2[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) m2[q] = mom[q * nc + ic];
  for (int v = warp; v < 5; v += kReconWarps) {
    R a[9];
#pragma unroll
    for (int n = 0; n < 9; ++n) a[n] = sh.a[n][v][lane];
    // |l| = 1 terms: cell means of the squared first derivatives (linear in the scaled
    // coordinates y, second moments m2); |l| = 2 terms: squared second derivatives
    const R gx[3] = {R(2) * a[3], a[6], a[7]};
    const R gy[3] = {a[6], R(2) * a[4], a[8]};
    const R gz[3] = {a[7], a[8], R(2) * a[5]};
    auto qf = [&](const R g[3]) {
      return m2[0] * g[0] * g[0] + m2[1] * g[1] * g[1] + m2[2] * g[2] * g[2] +
             R(2) * (m2[3] * g[0] * g[1] + m2[4] * g[0] * g[2] + m2[5] * g[1] * g[2]);
    };
    const R beta0 = a[0] * a[0] + a[1] * a[1] + a[2] * a[2] + qf(gx) + qf(gy) + qf(gz) +
                    R(4) * (a[3] * a[3] + a[4] * a[4] + a[5] * a[5]) + a[6] * a[6] + a[7] * a[7] +
                    a[8] * a[8];
    R tau = R(0);
    for (int s = 0; s < M; ++s) tau += fabs(beta0 - sh.bet[s][v][lane]);
    tau /= R(M);
    auto weight = [&](R gam, R bb) {
      const R r = tau / (bb + weps);
      R pw = r;
      for (int q = 1; q < wpow; ++q) pw *= r;
      return gam * (R(1) + pw);
    };
    const R w0 = weight(g0, beta0);
    R sum = w0;
    for (int s = 0; s < M; ++s) {
      const R w = weight(wg, sh.bet[s][v][lane]);
      sh.bet[s][v][lane] = w;
      sum += w;
    }
    const R is = R(1) / sum;
    const R wb0 = w0 * is;
    const R corr = wb0 * wg / g0;
#pragma unroll
    for (int s = 0; s < kMaxSub; ++s)
      sh.bet[s][v][lane] = s < M ? sh.bet[s][v][lane] * is - corr : R(0);
    sh.ca[v][lane] = wb0 / g0;
  }
  __syncthreads();

  // phase 4: linear part of the combination and the output, one variable per warp
  const R ih = R(1) / hcell[ic], ih2 = ih * ih;
  for (int v = warp; v < 5; v += kReconWarps) {
    R cl[3] = {R(0), R(0), R(0)};
    for (int s = 0; s < M; ++s) {
      const R f = sh.bet[s][v][lane];
#pragma unroll
      for (int t = 0; t < 3; ++t) cl[t] += f * sh.b[s][t][v][lane];
    }
    const R ca = sh.ca[v][lane];
    R C[9];
#pragma unroll
    for (int n = 0; n < 9; ++n) C[n] = ca * sh.a[n][v][lane];
    C[0] += cl[0];
    C[1] += cl[1];
    C[2] += cl[2];
    if (valid) {
      // Q = c0 + c1 dx + c2 dy + c3 dz + c4 dx^2 + c5 dy^2 + c6 dz^2 + c7 dxdy + c8 dxdz + c9 dydz
      const R shift = C[3] * m2[0] + C[4] * m2[1] + C[5] * m2[2] + C[6] * m2[3] +
                      C[7] * m2[4] + C[8] * m2[5];
      R* o = poly + (int64_t)kPolyStride * i + 10 * v;
      o[0] = c0.value_minus(v, shift);
      o[1] = C[0] * ih;
      o[2] = C[1] * ih;
      o[3] = C[2] * ih;
#pragma unroll
      for (int n = 3; n < 9; ++n) o[n + 1] = C[n] * ih2;
    }
  }
}

// Coefficient accessor of one cell's polynomial (kPolyStride values per cell).
template <class R>
struct PolyRef {
  const R* __restrict__ p;
  __device__ __forceinline__ R operator()(int v, int j) const { return __ldg(p + 10 * v + j); }
};

// ------------------------------------------------------------------------------------------
// Flux: four consecutive threads per face, one per Gauss point. Each evaluates both sides'
// reconstructions, rotates into the local frame (n1 normal, n2 = n1 x e_k normalised with e_k
// the axis least aligned with n1, n3 = n1 x n2), computes F^n and dF/dt, rotates back and
// weights by the quadrature weight; the four are summed with shuffles and written once.
template <class R>
__global__ void __launch_bounds__(128, sizeof(R) == 4 ? 4 : 1) k_flux(
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
      dl[a] = __ldcs(fgp + a * stride + gid);
      dr[a] = __ldcs(fgp + (3 + a) * stride + gid);
      n1[a] = __ldcs(fgp + (6 + a) * stride + gid);
    }
    const R w = __ldcs(fgp + 9 * stride + gid);
    R vl[5], gl[5][3], vr[5], gr[5][3];
    eval_poly(PolyRef<R>{poly + (int64_t)kPolyStride * o}, dl, vl, gl);
    if (nb >= 0) {
      eval_poly(PolyRef<R>{poly + (int64_t)kPolyStride * nb}, dr, vr, gr);
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
    R* o = fface + (int64_t)kFaceStride * f;
#pragma unroll
    for (int q = 0; q < 10; ++q) o[q] = acc[q];
  }
}


template <class R>
__device__ __forceinline__ bool physical(const double q[5], double gamma) {
  const double ke = 0.5 * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]) / q[0];
  const double p = (gamma - 1.0) * (q[4] - ke);
  return q[0] > 0.0 && p > 0.0;
}

// Sum of the signed face fluxes of one cell (the owner loses the outward flux), in the cell's
// fixed face order. FP64 path: FP64 sums. FP32 path: each component is accumulated as an
// unevaluated pair hi + lo of floats with the error-free TwoSum (Knuth), so the sum is exact to
// about 2^-48 relative without FP64 arithmetic (GB300 runs FP64 at 1/64 of the FP32 rate).
template <class R>
__device__ __forceinline__ void face_sums(int k0, int k1, const int32_t* __restrict__ cf_idx,
                                          const R* __restrict__ fface, double s[10]);
template <>
__device__ __forceinline__ void face_sums<double>(int k0, int k1, const int32_t* __restrict__ cf_idx,
                                                  const double* __restrict__ fface, double s[10]) {
#pragma unroll
  for (int q = 0; q < 10; ++q) s[q] = 0.0;
  for (int k = k0; k < k1; ++k) {
    const int32_t e = __ldg(cf_idx + k);
    const double* fp = fface + (int64_t)kFaceStride * (e >> 1);
    const double sg = (e & 1) ? 1.0 : -1.0;
#pragma unroll
    for (int q = 0; q < 10; ++q) s[q] += sg * __ldg(fp + q);
  }
}
template <>
__device__ __forceinline__ void face_sums<float>(int k0, int k1, const int32_t* __restrict__ cf_idx,
                                                 const float* __restrict__ fface, double s[10]) {
  float hi[10], lo[10];
#pragma unroll
  for (int q = 0; q < 10; ++q) hi[q] = lo[q] = 0.f;
  for (int k = k0; k < k1; ++k) {
    const int32_t e = __ldg(cf_idx + k);
    const float4* fp = reinterpret_cast<const float4*>(fface + (int64_t)kFaceStride * (e >> 1));
    const float4 a = __ldg(fp), b = __ldg(fp + 1), c = __ldg(fp + 2);
    float x[10] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y};
    const bool neg = !(e & 1);
#pragma unroll
    for (int q = 0; q < 10; ++q) {
      const float xv = neg ? -x[q] : x[q];
      const float t = __fadd_rn(hi[q], xv);
      const float bb = __fsub_rn(t, hi[q]);
      const float err = __fadd_rn(__fsub_rn(hi[q], __fsub_rn(t, bb)), __fsub_rn(xv, bb));
      hi[q] = t;
      lo[q] = __fadd_rn(lo[q], err);
    }
  }
#pragma unroll
  for (int q = 0; q < 10; ++q) s[q] = (double)hi[q] + (double)lo[q];
}

// Per cell: L = -(1/|Omega|) sum_f s_f F_f in the cell's fixed face order, then the
// requested update; the stage kernels also write the gather copy of the state they produce.
template <class R>
__global__ void __launch_bounds__(256) k_gather(
    int64_t nc, const int32_t* __restrict__ cf_ptr, const int32_t* __restrict__ cf_idx,
    const R* __restrict__ fface, const double* __restrict__ vol, int mode, double dt, double gamma,
    double* __restrict__ L, double* __restrict__ Lt, double* __restrict__ Qn,
    double* __restrict__ Qs, R* __restrict__ QA, R* __restrict__ QsA, int* flag) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nc) return;
  double s[10];
  face_sums(cf_ptr[i], cf_ptr[i + 1], cf_idx, fface, s);
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
    Gq<R>::store(QsA, i, q);
  } else {
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      q[v] = Qn[v * nc + i] + dt * L[v * nc + i] +
             (dt * dt / 6.0) * (Lt[v * nc + i] + 2.0 * lt[v]);
      Qn[v * nc + i] = q[v];
    }
    Gq<R>::store(QA, i, q);
  }
  if (!physical<R>(q, gamma)) atomicOr(flag, kErrNonphysical);
}

template <class R>
__global__ void k_permute_in(int64_t nc, const int32_t* __restrict__ perm,
                             const double* __restrict__ src, double* __restrict__ dst, R* gq) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nc) return;
  const int64_t c = perm[i];
  double q[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    q[v] = src[v * nc + c];
    dst[v * nc + i] = q[v];
  }
  if (gq) Gq<R>::store(gq, i, q);
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
void launch_recon(const DevMesh& m, const GeoR<R>& g, const KParams<R>& p, const R* QA,
                  R* poly, cudaStream_t st) {
  const size_t smem = sizeof(ReconShared<R>) + (size_t)m.kmax * 5 * kTile * sizeof(R);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_recon<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_recon<R><<<(unsigned)m.n_tiles, kReconThreads, smem, st>>>(
      m.nc, QA, m.t_K, m.t_cnt, m.t_st, m.t_sb, m.t_idx, m.n_sub, g.Ap, g.Bp, g.mom, g.h,
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
  fp.pr_fix = p.pr_fix;
  k_flux<R><<<blocks_for(4 * m.nf, 128), 128, 0, st>>>(m.nf, m.nc, m.f_owner, m.f_nb, m.f_wall,
                                                         g.fgp, poly, fp, (R)dt, fface, flag);
}
template <class R>
void launch_gather(const DevMesh& m, const Geo64& g, const R* fface, int mode, double dt,
                   double gamma, double* L, double* Lt, double* Qn, double* Qs, R* QA, R* QsA,
                   int* flag, cudaStream_t st) {
  k_gather<R><<<blocks_for(m.nc, 256), 256, 0, st>>>(m.nc, m.cf_ptr, m.cf_idx, fface, g.vol, mode,
                                                       dt, gamma, L, Lt, Qn, Qs, QA, QsA, flag);
}
template <class R>
void launch_permute_in(int64_t nc, const int32_t* perm, const double* src, double* dst, R* gq,
                       cudaStream_t st) {
  k_permute_in<R><<<blocks_for(nc, 256), 256, 0, st>>>(nc, perm, src, dst, gq);
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
template void launch_permute_in<double>(int64_t, const int32_t*, const double*, double*, double*,
                                        cudaStream_t);
template void launch_permute_in<float>(int64_t, const int32_t*, const double*, double*, float*,
                                       cudaStream_t);
template void launch_recon<float>(const DevMesh&, const GeoR<float>&, const KParams<float>&,
                                  const float*, float*, cudaStream_t);
template void launch_flux<double>(const DevMesh&, const GeoR<double>&, const KParams<double>&,
                                  const double*, double, double*, int*, cudaStream_t);
template void launch_flux<float>(const DevMesh&, const GeoR<float>&, const KParams<float>&,
                                 const float*, double, float*, int*, cudaStream_t);
template void launch_gather<double>(const DevMesh&, const Geo64&, const double*, int, double, double,
                                    double*, double*, double*, double*, double*, double*, int*,
                                    cudaStream_t);
template void launch_gather<float>(const DevMesh&, const Geo64&, const float*, int, double, double,
                                   double*, double*, double*, double*, float*, float*, int*,
                                   cudaStream_t);

}  // namespace gks

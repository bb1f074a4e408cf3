// Hot-path kernels: WENO reconstruction per cell (Section 2), gas-kinetic flux per face Gauss
// point (Section 3.2), per-cell gather of face fluxes with the two-stage fourth-order update
// (Section 3.3), the time-step bound, and caller-order permutations.
#include <cuda_runtime.h>

#include <cfloat>
#include <cmath>
#include <type_traits>

#include "gks_device.cuh"
#include "gks_ff.cuh"
#include "gks_kinetic.cuh"
#include "gks_flux_f32x2.cuh"

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
  __device__ static void store_ff(float* QA, int64_t c, const ff q[5]) {
    float4* p = reinterpret_cast<float4*>(QA + 12 * c);
    p[0] = make_float4(q[0].h, q[1].h, q[2].h, q[3].h);
    p[1] = make_float4(q[4].h, q[0].l, q[1].l, q[2].l);
    p[2] = make_float4(q[3].l, q[4].l, 0.f, 0.f);
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

// FP64 value of variable v of a gather copy.
__device__ __forceinline__ double unpack_value(const Gq<float>& g, int v) {
  return (double)g.hi[v] + (double)g.lo[v];
}
__device__ __forceinline__ double unpack_value(const Gq<double>& g, int v) { return g.q[v]; }

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
// Asynchronous bulk copies global -> shared completed on an mbarrier (transaction bytes), and a
// bounded wait on it.
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// bytes: a multiple of 16; dst and src 16-byte aligned
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes,
                                          uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// Bulk store shared -> global in a bulk group (src and dst 16-byte aligned, bytes a multiple of
// 16). The threads that wrote the source with ordinary stores fence them into the async proxy
// (fence_proxy_async_shared) and the block synchronises before one thread issues the store;
// that thread waits until the store has read its source before the block's shared memory may
// be reused.
__device__ __forceinline__ void fence_proxy_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void bulk_store(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
               "r"(smem_u32(src)), "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void bulk_store_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Each try_wait suspends the thread for at most a hardware time limit; the loop gives up after
// `tries` attempts (by default kWaitTries, far beyond the microseconds a tile's copies take).
constexpr int kWaitTries = 1 << 22;
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int tries) {
  for (int it = 0; it < tries; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// ------------------------------------------------------------------------------------------
// Reconstruction, one block of five warps per 32-cell tile (lane = cell). For each conserved
// variable v of each cell:
//   dq_k = Q_k - Q_0 over the big stencil                      (phase 1, all warps, to shared)
//   a    = A+ dq   (quadratic P0, 9 coefficients in centred scaled coordinates) and
//   b_m  = B_m dq|S_m (linear P_m) with beta_m (Eq. indicator); rows and sub-stencils are
//   spread over the warps                                                            (phase 2)
//   beta_0, tau, omega, omega-bar (Section 2), one variable per warp               (phase 3)
//   C = (wb_0/g_0) a + sum_m (wb_m - wb_0 g_m/g_0) b_m, i.e. Eq. weno as one polynomial (phase 4)
// Output: 10 coefficients per variable of the polynomial in physical offsets from the centroid.
// With kPf, when the block starts, the tile's pseudo-inverse rows (a contiguous block of the
// interleaved layout) are prefetched into L2 by a bulk prefetch, and the sub-stencil entries are
// either copied into shared memory by a bulk copy on an mbarrier (kStB: where that costs the
// range no resident blocks) or prefetched into L2 as well, so that the transfers overlap phase
// 1; phase 2 then reads the rows from L2 (each row once, two rows per warp in one member loop,
// so that two independent loads per member are in flight) and the entries from shared memory or
// L2. Without kPf phase 2 reads both from global memory. Staging the rows in shared memory
// as well (they are read once, so the staging bought only the overlap) held the range's blocks
// to 2-3 per SM: 0.669 against 0.598 ms per FP32 pass on the 64^3-cube mesh with the enlarged
// stencils, 6.54 against 5.38 ms in FP64.
constexpr int kReconWarps = 5;
constexpr int kReconThreads = kReconWarps * kTile;
constexpr int kReconBlocksPerSM = 5;  // the register bound (launch bounds) of k_recon

// Shared-memory layout of one block for a range with largest stencil Kr, largest sum of
// sub-stencil member counts Sr and largest number of sub-stencil slots Mr, in units of one
// interleaved row (kTile values): [mbarrier, 16 B][B entries 4 Sr] (only with kPf and stb: the
// sub-stencil entries staged by a bulk copy), then a[9][5], b[Mr][3][5], beta[Mr][5], dq[Kr][5]
// (the last in the lane-major form of DqRow below). Every part starts on a 16-byte boundary.
// (a_off marks where staged rows would start; the rows come through L2.)

template <class R>
struct ReconSmem {
  size_t a_off, b_off, ca_off, cb_off, cbet_off, dq_off, bytes;
  __host__ __device__ ReconSmem(int Kr, int Sr, int Mr, bool pf, bool stb) {
    const size_t row = (size_t)kTile * sizeof(R);
    a_off = pf ? 16 : 0;
    b_off = a_off;
    ca_off = b_off + (pf && stb ? 4 * (size_t)Sr * row : 0);
    cb_off = ca_off + 45 * row;
    cbet_off = cb_off + 15 * (size_t)Mr * row;
    dq_off = cbet_off + 5 * (size_t)Mr * row;
    // the dq region holds the tile's output records [lane][kPolyStride] once phase 2 is done
    bytes = dq_off + (5 * (size_t)Kr > (size_t)kPolyStride ? 5 * (size_t)Kr : kPolyStride) * row;
  }
};

// Stencil differences in shared memory: variables 0-3 of member k as 16-byte vectors with the
// lane fastest ([k][h][lane], h < 1 in FP32, h < 2 in FP64), variable 4 in a plain row [k][lane]
// after all of them, so that a thread reads or writes a member's five differences in two (FP32)
// or three (FP64) shared-memory accesses instead of five; consecutive lanes touch consecutive
// 16-byte words (no bank conflicts). Against five scalar rows: 0.599 -> 0.595 ms per FP32 pass
// on the 64^3-cube mesh.
template <class R>
struct DqRow;
template <>
struct DqRow<float> {
  __device__ __forceinline__ static void put(unsigned char* s, int k, int lane, const float d[4]) {
    reinterpret_cast<float4*>(s)[k * kTile + lane] = make_float4(d[0], d[1], d[2], d[3]);
  }
  __device__ __forceinline__ static void get(const unsigned char* s, int k, int lane, float d[4]) {
    const float4 x = reinterpret_cast<const float4*>(s)[k * kTile + lane];
    d[0] = x.x; d[1] = x.y; d[2] = x.z; d[3] = x.w;
  }
};
template <>
struct DqRow<double> {
  __device__ __forceinline__ static void put(unsigned char* s, int k, int lane, const double d[4]) {
    double2* p = reinterpret_cast<double2*>(s) + 2 * k * kTile + lane;
    p[0] = make_double2(d[0], d[1]);
    p[kTile] = make_double2(d[2], d[3]);
  }
  __device__ __forceinline__ static void get(const unsigned char* s, int k, int lane, double d[4]) {
    const double2* p = reinterpret_cast<const double2*>(s) + 2 * k * kTile + lane;
    const double2 x = p[0], y = p[kTile];
    d[0] = x.x; d[1] = x.y; d[2] = y.x; d[3] = y.y;
  }
};

// One sub-stencil entry (three pseudo-inverse coefficients and the member index) of one lane:
// one 16-byte load in FP32, two in FP64, from shared memory (staged) or through the read-only
// path (global). Against four interleaved rows: 0.571 -> 0.569 ms per FP32 pass.
template <class R>
struct BRec;
template <>
struct BRec<float> {
  __device__ __forceinline__ static void get(const float* e, bool staged, float c[4]) {
    const float4* p = reinterpret_cast<const float4*>(e);
    const float4 x = staged ? *p : __ldg(p);
    c[0] = x.x; c[1] = x.y; c[2] = x.z; c[3] = x.w;
  }
};
template <>
struct BRec<double> {
  __device__ __forceinline__ static void get(const double* e, bool staged, double c[4]) {
    const double2* p = reinterpret_cast<const double2*>(e);
    const double2 x = staged ? p[0] : __ldg(p), y = staged ? p[1] : __ldg(p + 1);
    c[0] = x.x; c[1] = x.y; c[2] = y.x; c[3] = y.y;
  }
};

// A variable's ten output coefficients as five 8-byte (FP32) or 16-byte (FP64) shared stores
// (a record of kPolyStride values starts on a 16-byte boundary; variable v at 10 v values).
template <class R>
struct PolyPair;
template <>
struct PolyPair<float> {
  __device__ __forceinline__ static void put(float* so, const float o[10]) {
    float2* p = reinterpret_cast<float2*>(so);
#pragma unroll
    for (int j = 0; j < 5; ++j) p[j] = make_float2(o[2 * j], o[2 * j + 1]);
  }
};
template <>
struct PolyPair<double> {
  __device__ __forceinline__ static void put(double* so, const double o[10]) {
    double2* p = reinterpret_cast<double2*>(so);
#pragma unroll
    for (int j = 0; j < 5; ++j) p[j] = make_double2(o[2 * j], o[2 * j + 1]);
  }
};

// Quotients of the weights and the output scaling: the FP32 path uses the fast division
// intrinsic (x times an approximate reciprocal, within 2 ulp for divisors below 2^126: the
// indicators, weights and cell sizes here), the FP64 path the IEEE division. Against IEEE
// divisions in FP32: 0.436 -> 0.417 ms per pass on the 64^3-cube mesh (the weights of phase 3
// take about a dozen quotients per thread).
template <class R>
__device__ __forceinline__ R wdiv(R a, R b) {
  return a / b;
}
template <>
__device__ __forceinline__ float wdiv<float>(float a, float b) {
  return __fdividef(a, b);
}

// Five resident blocks per SM as the register bound (at most 80 registers a thread; 72 used):
// on the 64^3-cube hybrid mesh with the enlarged stencils 0.598 ms per FP32 pass, 0.611 ms at 6
// blocks (64 registers, spills); before the rows went through L2, 0.664 ms against 0.697 ms
// unbounded (4 blocks).
// A uniform range (every tile with the same stencil size K and sub-stencil counts cnt): the
// tile's offsets into the interleaved arrays are st0 + K (tile - tile0) and sb0 + S (tile - tile0),
// so no table load stands between the block's start and its first stencil gathers.
struct ReconUni {
  int on, K, S;
  uint64_t cnt;
  int64_t st0, sb0;
};

template <class R, bool kPf, bool kStB>
__global__ void __launch_bounds__(kReconThreads, kReconBlocksPerSM) k_recon(
    int64_t nc, int64_t tile0, int Kr, int Sr, int Mr, ReconUni u, const R* __restrict__ QA,
    const int32_t* __restrict__ t_K, const uint64_t* __restrict__ t_cnt,
    const int32_t* __restrict__ t_st, const int32_t* __restrict__ t_sb,
    const int32_t* __restrict__ t_idx, const int8_t* __restrict__ n_sub,
    const R* __restrict__ Ap, const R* __restrict__ Bp, const R* __restrict__ mom,
    const R* __restrict__ hcell, R wg, R weps, int wpow, R* __restrict__ poly, int* flag,
    int wait_tries, int withhold) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const ReconSmem<R> L(Kr, Sr, Mr, kPf, kStB);
  R* sa = reinterpret_cast<R*>(smem_raw + L.ca_off);      // [n][v][lane]
  R* sb = reinterpret_cast<R*>(smem_raw + L.cb_off);      // [m][t][v][lane]
  R* sbet = reinterpret_cast<R*>(smem_raw + L.cbet_off);  // [m][v][lane]
  unsigned char* sdqv = smem_raw + L.dq_off;              // variables 0-3, DqRow<R>
  R* sdq4 = reinterpret_cast<R*>(sdqv + 4 * (size_t)Kr * kTile * sizeof(R));  // [k][lane]
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  const int64_t tile = tile0 + blockIdx.x;
  const int lane = threadIdx.x & (kTile - 1);
  const int warp = threadIdx.x / kTile;
  const int64_t tl = tile - tile0;
  const int K = u.on ? u.K : __ldg(t_K + tile);
  const uint64_t cnt = u.on ? u.cnt : __ldg(t_cnt + tile);
  const int64_t st = u.on ? u.st0 + tl * u.K : (int64_t)__ldg(t_st + tile);
  const int64_t sbo = u.on ? u.sb0 + tl * u.S : (int64_t)__ldg(t_sb + tile);
  const R* Ag = Ap + st * 9 * kTile;
  const R* Bg = Bp + sbo * 4 * kTile;
  int S = 0, Mt = 0;  // entries and sub-stencil slots of this tile
#pragma unroll
  for (int q = 0; q < kMaxSub; ++q) {
    const int c = (int)((cnt >> (8 * q)) & 0xffu);
    S += c;
    if (c) Mt = q + 1;
  }
  if (kPf) {
    if (threadIdx.x == 0) {
      mbar_init(bar);
      const uint32_t ab = 9u * K * kTile * sizeof(R), bb = 4u * S * kTile * sizeof(R);
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" :: "l"(Ag), "r"(ab) : "memory");
      if (!kStB && bb)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" :: "l"(Bg), "r"(bb) : "memory");
      // withhold != 0 (the timeout test of gks_debug_recon_wait): no copy is issued and 16
      // bytes more than the copies would bring are expected, so the barrier's phase never
      // completes and the bounded wait below runs out with nothing in flight
      mbar_expect_tx(bar, (kStB ? bb : 0u) + (withhold ? 16u : 0u));
      if (kStB && bb && !withhold) bulk_load(smem_raw + L.b_off, Bg, bb, bar);
    }
  }
  const int64_t i = tile * kTile + lane;
  const bool valid = i < nc;
  const int64_t ic = valid ? i : tile * kTile;  // padded lanes mirror the tile's first cell
  // per-cell data of the later phases: the moments and the cell size are prefetched into L2 now
  // and loaded in phase 3 (held in registers through phases 1 and 2 they cost spills: 0.437
  // against 0.470 ms per FP32 pass on the 64^3-cube mesh with the uniform-range offsets, 0.456
  // against 0.457 without them)
  const int M = n_sub[ic];
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < 6; ++q)
      asm volatile("prefetch.global.L2 [%0];" ::"l"(mom + q * nc + ic));
    asm volatile("prefetch.global.L2 [%0];" ::"l"(hcell + ic));
  }
  const int32_t* sidx = t_idx + st * kTile + lane;
  Gq<R> c0;
  c0.load(QA, ic);
  if (kPf) __syncthreads();  // the barrier is initialised before anyone waits on it

  // phase 1: stencil differences, members split over the warps, four per batch: all index
  // loads, then all state loads, then the differences
  for (int k0 = warp; k0 < K; k0 += 4 * kReconWarps) {
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
      R d[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) d[v] = g[u].minus(c0, v);
      DqRow<R>::put(sdqv, k, lane, d);
      sdq4[k * kTile + lane] = g[u].minus(c0, 4);
    }
  }
  const R* A;
  const R* Bt;
  if (kPf) {
    // every thread waits for the copies; a block whose wait ran out reports it and stops
    const int tries = wait_tries > 0 ? wait_tries : kWaitTries;
    bool ok = mbar_wait(bar, 0, tries);
    if (!ok) ok = mbar_wait(bar, 0, tries);  // let copies still in flight land before leaving
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) atomicOr(flag, kErrTimeout);
      return;
    }
    A = Ag + lane;
    Bt = (kStB ? reinterpret_cast<const R*>(smem_raw + L.b_off) : Bg) + 4 * lane;
  } else {
    __syncthreads();
    A = Ag + lane;
    Bt = Bg + 4 * lane;
  }

  // phase 2: rows n = warp, warp + 5 of a = A+ dq (both in one member loop: each stencil
  // difference is read once for the two rows), and the sub-stencil fits b_m with their
  // indicators beta_m = |b_m|^2 (scaled coordinates); sub-stencils go to the warps in reverse
  // order (m = 4 - warp, 9 - warp) so that the warp with one row takes two of them
  {
    const int n0 = warp, n1 = warp + kReconWarps;
    const bool two = n1 < 9;
    const int n1c = two ? n1 : n0;
    R acc0[5] = {R(0), R(0), R(0), R(0), R(0)}, acc1[5] = {R(0), R(0), R(0), R(0), R(0)};
#pragma unroll 6
    for (int k = 0; k < K; ++k) {
      const R r0 = __ldg(A + (9 * k + n0) * kTile);
      const R r1 = __ldg(A + (9 * k + n1c) * kTile);
      R d[5];
      DqRow<R>::get(sdqv, k, lane, d);
      d[4] = sdq4[k * kTile + lane];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        acc0[v] += r0 * d[v];
        acc1[v] += r1 * d[v];
      }
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      sa[(5 * n0 + v) * kTile + lane] = acc0[v];
      if (two) sa[(5 * n1 + v) * kTile + lane] = acc1[v];
    }
  }
  for (int s = kReconWarps - 1 - warp; s < Mt; s += kReconWarps) {
    int slot = 0;
    for (int q = 0; q < s; ++q) slot += (int)((cnt >> (8 * q)) & 0xffu);
    const int cs = (int)((cnt >> (8 * s)) & 0xffu);
    const R* e = Bt + (int64_t)4 * kTile * slot;
    R b[3][5];
#pragma unroll
    for (int t = 0; t < 3; ++t)
#pragma unroll
      for (int v = 0; v < 5; ++v) b[t][v] = R(0);
#pragma unroll 2
    for (int j = 0; j < cs; ++j, e += 4 * kTile) {
      R c[4];
      BRec<R>::get(e, kPf && kStB, c);
      const int k = (int)c[3];
      R dq[5];
      DqRow<R>::get(sdqv, k, lane, dq);
      dq[4] = sdq4[k * kTile + lane];
#pragma unroll
      for (int v = 0; v < 5; ++v)
#pragma unroll
        for (int t = 0; t < 3; ++t) b[t][v] += c[t] * dq[v];
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      sbet[(5 * s + v) * kTile + lane] = b[0][v] * b[0][v] + b[1][v] * b[1][v] + b[2][v] * b[2][v];
#pragma unroll
      for (int t = 0; t < 3; ++t) sb[((3 * s + t) * 5 + v) * kTile + lane] = b[t][v];
    }
  }
  __syncthreads();

  // phase 3: nonlinear weights, variable v = warp
  R m2[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) m2[q] = mom[q * nc + ic];
  const R hc = hcell[ic];
  const R g0 = R(1) - wg * R(M);
  const int v = warp;
  {
    R a[9];
#pragma unroll
    for (int n = 0; n < 9; ++n) a[n] = sa[(5 * n + v) * kTile + lane];
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
    for (int s = 0; s < M; ++s) tau += fabs(beta0 - sbet[(5 * s + v) * kTile + lane]);
    tau = wdiv(tau, R(M));
    auto weight = [&](R gam, R bb) {
      const R r = wdiv(tau, bb + weps);
      R pw = r;
      for (int q = 1; q < wpow; ++q) pw *= r;
      return gam * (R(1) + pw);
    };
    const R w0 = weight(g0, beta0);
    R sum = w0;
    R wm[kMaxSub];
#pragma unroll
    for (int s = 0; s < kMaxSub; ++s) {
      wm[s] = s < M ? weight(wg, sbet[(5 * s + v) * kTile + lane]) : R(0);
      sum += wm[s];
    }
    const R is = wdiv(R(1), sum);
    const R wb0 = w0 * is;
    const R ig0 = wdiv(R(1), g0);
    const R corr = wb0 * wg * ig0;
    // phase 4 (same warp, same variable): linear part of the combination and the output
    R cl[3] = {R(0), R(0), R(0)};
#pragma unroll
    for (int s = 0; s < kMaxSub; ++s) {
      if (s < M) {
        const R f = wm[s] * is - corr;
#pragma unroll
        for (int t = 0; t < 3; ++t) cl[t] += f * sb[((3 * s + t) * 5 + v) * kTile + lane];
      }
    }
    const R ca = wb0 * ig0;
    R C[9];
#pragma unroll
    for (int n = 0; n < 9; ++n) C[n] = ca * a[n];
    C[0] += cl[0];
    C[1] += cl[1];
    C[2] += cl[2];
    {
      const R ih = wdiv(R(1), hc), ih2 = ih * ih;
      // Q = c0 + c1 dx + c2 dy + c3 dz + c4 dx^2 + c5 dy^2 + c6 dz^2 + c7 dxdy + c8 dxdz + c9 dydz
      const R shift = C[3] * m2[0] + C[4] * m2[1] + C[5] * m2[2] + C[6] * m2[3] +
                      C[7] * m2[4] + C[8] * m2[5];
      R o[10];
      o[0] = R(0);  // c0's component v, selected without a dynamic register index
#pragma unroll
      for (int q = 0; q < 5; ++q)
        if (q == v) o[0] = c0.value_minus(q, shift);
      o[1] = C[0] * ih;
      o[2] = C[1] * ih;
      o[3] = C[2] * ih;
#pragma unroll
      for (int n = 3; n < 9; ++n) o[n + 1] = C[n] * ih2;
      // the tile's output records go to shared memory (the stencil differences are dead after
      // phase 2) and leave in one contiguous bulk store: written directly, every store of a
      // warp touched 32 sectors for 4 bytes each (0.569 -> 0.457 ms per FP32 pass on the
      // 64^3-cube mesh, 5.36 -> 5.34 ms in FP64)
      R* so = reinterpret_cast<R*>(smem_raw + L.dq_off) + lane * kPolyStride + 10 * v;
      PolyPair<R>::put(so, o);
    }
  }
  fence_proxy_async_shared();
  __syncthreads();
  if (threadIdx.x == 0) {
    const int64_t nv = nc - tile * kTile < kTile ? nc - tile * kTile : kTile;
    bulk_store(poly + (int64_t)kPolyStride * tile * kTile, smem_raw + L.dq_off,
               (uint32_t)(nv * kPolyStride * sizeof(R)));
    bulk_store_wait_read();
  }
}

// Coefficient accessor of one cell's polynomial (kPolyStride values per cell).
template <class R>
struct PolyRef {
  const R* __restrict__ p;
  __device__ __forceinline__ R operator()(int v, int j) const { return __ldg(p + 10 * v + j); }
};
// A variable's ten coefficients as five pair loads (a cell's record starts on a 16-byte
// boundary: kPolyStride values of 4 or 8 bytes; variable v at 10 v values).
// In FP32 a variable's ten coefficients start on a 16-byte boundary for even v and on an 8-byte
// one for odd v: three loads (16 + 16 + 8 or 8 + 16 + 16 bytes) instead of five.
__device__ __forceinline__ void load_coefs(const PolyRef<float>& c, int v, float k[10]) {
  const float* p = c.p + 10 * v;
  if ((v & 1) == 0) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(p));
    const float4 b = __ldg(reinterpret_cast<const float4*>(p + 4));
    const float2 d = __ldg(reinterpret_cast<const float2*>(p + 8));
    k[0] = a.x; k[1] = a.y; k[2] = a.z; k[3] = a.w;
    k[4] = b.x; k[5] = b.y; k[6] = b.z; k[7] = b.w;
    k[8] = d.x; k[9] = d.y;
  } else {
    const float2 a = __ldg(reinterpret_cast<const float2*>(p));
    const float4 b = __ldg(reinterpret_cast<const float4*>(p + 2));
    const float4 d = __ldg(reinterpret_cast<const float4*>(p + 6));
    k[0] = a.x; k[1] = a.y;
    k[2] = b.x; k[3] = b.y; k[4] = b.z; k[5] = b.w;
    k[6] = d.x; k[7] = d.y; k[8] = d.z; k[9] = d.w;
  }
}
__device__ __forceinline__ void load_coefs(const PolyRef<double>& c, int v, double k[10]) {
  const double2* q = reinterpret_cast<const double2*>(c.p + 10 * v);
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const double2 t = __ldg(q + i);
    k[2 * i] = t.x;
    k[2 * i + 1] = t.y;
  }
}

// Positivity fallback at a Gauss point (off unless the solver asks for it; the paper prints no
// positivity treatment): a side whose reconstructed state has rho <= 0 or p <= 0 (or NaN) takes
// the cell average of its cell, read from the gather copy the reconstruction used, with a zero
// gradient. p > 0 is tested as rho E > |m|^2 / 2, which needs no division.
template <class R>
__device__ __forceinline__ void first_order_if_nonphysical(const R* __restrict__ QA, int64_t c,
                                                           R v[5], R g[5][3]) {
  const R m2 = v[1] * v[1] + v[2] * v[2] + v[3] * v[3];
  if (v[0] > R(0) && v[0] * v[4] > R(0.5) * m2) return;
  Gq<R> q;
  q.load(QA, c);
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    v[k] = q.value(k);
#pragma unroll
    for (int a = 0; a < 3; ++a) g[k][a] = R(0);
  }
}

// ------------------------------------------------------------------------------------------
// Flux: four consecutive threads per face, one per Gauss point. Each evaluates both sides'
// reconstructions, rotates into the local frame (n1 normal, n2 = n1 x e_k normalised with e_k
// the axis least aligned with n1, n3 = n1 x n2), computes F^n and dF/dt, rotates back and
// weights by the quadrature weight; the four are summed with shuffles and written once.
// kFull selects the flux form and kTau0 a zero collision time at compile time, so that each
// instance carries only the arithmetic (and registers) of its own form. The FP32 instances do
// the two sides' work on packed f32x2 arithmetic (gp_flux_global2: the flux templates
// instantiated with the pair type P2). Resident blocks per SM, measured: smooth form 6 (0.442 ms
// per launch on the 64^3-cube mesh; 5 and 7 blocks 0.456 and 0.446; the scalar form at 7
// blocks 0.477); full form 4 (6.53 ms per launch on the 128^3-cube explosion; 3 and 5 blocks
// 6.99 and 7.44; the scalar form 7.06).
#ifndef GKS_FLUX_SMOOTH_MIN_BLOCKS
#define GKS_FLUX_SMOOTH_MIN_BLOCKS 6  // resident 128-thread blocks per SM, FP32 smooth flux
#endif
#ifndef GKS_FLUX_FULL_MIN_BLOCKS
#define GKS_FLUX_FULL_MIN_BLOCKS 4  // resident 128-thread blocks per SM, FP32 full flux
#endif
#ifndef GKS_FLUX_FP64_MIN_BLOCKS
#define GKS_FLUX_FP64_MIN_BLOCKS 1  // resident 128-thread blocks per SM, FP64 flux
#endif
// One 16-byte (FP32) or 32-byte (FP64) part of a face record of kFaceStride values: part j holds
// values 4j .. 4j + 3 of acc (values 10 and 11 are padding, written as zeros).
template <class R>
struct FaceRec;
template <>
struct FaceRec<float> {
  __device__ __forceinline__ static void put(float* rec, int j, const float acc[10]) {
    float4 x;
    if (j == 0) x = make_float4(acc[0], acc[1], acc[2], acc[3]);
    else if (j == 1) x = make_float4(acc[4], acc[5], acc[6], acc[7]);
    else x = make_float4(acc[8], acc[9], 0.f, 0.f);
    reinterpret_cast<float4*>(rec)[j] = x;
  }
};
template <>
struct FaceRec<double> {
  __device__ __forceinline__ static void put(double* rec, int j, const double acc[10]) {
    double2 x, y;
    if (j == 0) { x = make_double2(acc[0], acc[1]); y = make_double2(acc[2], acc[3]); }
    else if (j == 1) { x = make_double2(acc[4], acc[5]); y = make_double2(acc[6], acc[7]); }
    else { x = make_double2(acc[8], acc[9]); y = make_double2(0.0, 0.0); }
    double2* p = reinterpret_cast<double2*>(rec) + 2 * j;
    p[0] = x;
    p[1] = y;
  }
};

template <class R, bool kFull, bool kTau0>
__global__ void __launch_bounds__(128, sizeof(R) == 4 ? (kFull ? GKS_FLUX_FULL_MIN_BLOCKS : GKS_FLUX_SMOOTH_MIN_BLOCKS)
                                                      : GKS_FLUX_FP64_MIN_BLOCKS)
    k_flux(
    int64_t nf, int64_t nc, const int32_t* __restrict__ f_owner, const int32_t* __restrict__ f_nb,
    const int8_t* __restrict__ f_wall, const R* __restrict__ fgp, const R* __restrict__ poly,
    const R* __restrict__ QA, int fallback, FluxParams<R> P, const R* __restrict__ wall_tab, R dt,
    R* __restrict__ fface, int* flag) {
  P.full = kFull;
  if (kTau0) P.tau_model = 0;
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
    if (fallback) first_order_if_nonphysical(QA, o, vl, gl);
    if (nb >= 0) {
      eval_poly(PolyRef<R>{poly + (int64_t)kPolyStride * nb}, dr, vr, gr);
      if (fallback) first_order_if_nonphysical(QA, nb, vr, gr);
    } else {
      wall_ghost(P, wall, wall_data(wall_tab, wall), vl, gl, vr, gr);  // the wall's ghost
    }
    bool ok;
    if constexpr (sizeof(R) == 4)
      ok = gp_flux_global2(P, vl, gl, vr, gr, n1, w, dt, acc);  // both sides on packed f32x2
    else
      ok = gp_flux_global(P, vl, gl, vr, gr, n1, w, dt, acc);
    if (!ok) atomicOr(flag, kErrNonphysical);
  }
  // sum the four Gauss points of the face (lanes 4f .. 4f+3 of one warp)
#pragma unroll
  for (int q = 0; q < 10; ++q) {
    acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], 1);
    acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], 2);
  }
  // every lane of the face now holds the sums; lanes 4f + j, j < 3, write the record's 16-byte
  // part j (values 4j .. 4j + 3; the two padding values of part 2 are written as zeros), so a
  // warp writes its eight faces' 384 contiguous bytes in one store
  if (active && (gid & 3) < 3) {
    if (wall >= 0) wall_flux_fix(wall, wall_data(wall_tab, wall), acc);
    FaceRec<R>::put(fface + (int64_t)kFaceStride * f, (int)(gid & 3), acc);
  }
}

// rho > 0 and p > 0, the latter as rho E > |m|^2 / 2 (gamma > 1; no division; false for NaN).
__device__ __forceinline__ bool physical(const double q[5]) {
  const double m2 = q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
  return q[0] > 0.0 && q[0] * q[4] > 0.5 * m2;
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

// Per cell: L = -(1/|Omega|) sum_f s_f F_f in the cell's fixed face order, and Lt from dF/dt
// (the residual of gks_residual), in FP64.
template <class R>
__global__ void __launch_bounds__(256) k_gather(
    int64_t nc, const int32_t* __restrict__ cf_ptr, const int32_t* __restrict__ cf_idx,
    const R* __restrict__ fface, const double* __restrict__ ivol, double* __restrict__ L,
    double* __restrict__ Lt) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nc) return;
  double s[10];
  face_sums(cf_ptr[i], cf_ptr[i + 1], cf_idx, fface, s);
  const double iv = ivol[i];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    L[v * nc + i] = s[v] * iv;
    Lt[v * nc + i] = s[5 + v] * iv;
  }
}

// ------------------------------------------------------------------------------------------
// The two stages of the fourth-order update (Section 3.3) on the gather copy of the state,
// which is the solver state itself: FP64 path [q0..q4, 0] per cell; FP32 path the float-float
// pairs (hi, lo) of each variable. With the cell's face sums s (F^n part) and st (dF/dt part),
// L = s / |Omega|, Lt = st / |Omega|:
//   stage 1: keep L, Lt;           Q*      = Q^n + dt/2 L + dt^2/8 Lt
//   stage 2 (Lt* of Q*):           Q^{n+1} = Q^n + dt L + dt^2/6 (Lt + 2 Lt*)
// FP32 path: every operation in float-float arithmetic, so the update is conservative to about
// 2^-46 relative and issues no FP64 instruction.

// Face sums as float-float pairs, components q0..9 (FP32 path).
__device__ __forceinline__ void face_sums_ff(int k0, int k1, const int32_t* __restrict__ cf_idx,
                                             const float* __restrict__ fface, int q0, ff s[10]) {
#pragma unroll
  for (int q = 0; q < 10; ++q) s[q] = ff{0.f, 0.f};
  for (int k = k0; k < k1; ++k) {
    const int32_t e = __ldg(cf_idx + k);
    const float4* fp = reinterpret_cast<const float4*>(fface + (int64_t)kFaceStride * (e >> 1));
    const float4 a = __ldg(fp), b = __ldg(fp + 1), c = __ldg(fp + 2);
    const float x[10] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y};
    const bool neg = !(e & 1);
#pragma unroll
    for (int q = 0; q < 10; ++q) {
      if (q < q0) continue;
      const ff t = two_sum(s[q].h, neg ? -x[q] : x[q]);
      s[q] = ff{t.h, __fadd_rn(s[q].l, t.l)};
    }
  }
#pragma unroll
  for (int q = 0; q < 10; ++q) s[q] = two_sum(s[q].h, s[q].l);
}

template <bool kSecond>
__global__ void __launch_bounds__(256) k_stage_f(
    int64_t nc, const int32_t* __restrict__ cf_ptr, const int32_t* __restrict__ cf_idx,
    const float* __restrict__ fface, const ff* __restrict__ ivol, ff c1, ff c2,
    ff* __restrict__ L, ff* __restrict__ Lt, float* __restrict__ QA, float* __restrict__ QsA,
    int* flag) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nc) return;
  ff s[10];
  face_sums_ff(cf_ptr[i], cf_ptr[i + 1], cf_idx, fface, kSecond ? 5 : 0, s);
  const ff iv = ivol[i];
  Gq<float> g;
  g.load(QA, i);
  ff q[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    const ff qn{g.hi[v], g.lo[v]};
    const ff lt = ff_mul(s[5 + v], iv);
    if (!kSecond) {  // c1 = dt/2, c2 = dt^2/8
      const ff l = ff_mul(s[v], iv);
      L[v * nc + i] = l;
      Lt[v * nc + i] = lt;
      q[v] = ff_add(qn, ff_add(ff_mul(c1, l), ff_mul(c2, lt)));
    } else {  // c1 = dt, c2 = dt^2/6
      const ff lt2 = ff_add(Lt[v * nc + i], ff_twice(lt));
      q[v] = ff_add(qn, ff_add(ff_mul(c1, L[v * nc + i]), ff_mul(c2, lt2)));
    }
  }
  Gq<float>::store_ff(kSecond ? QA : QsA, i, q);
  // rho > 0 and rho E > |m|^2 / 2 on the leading parts (false for NaN)
  const float m2 = q[1].h * q[1].h + q[2].h * q[2].h + q[3].h * q[3].h;
  if (!(q[0].h > 0.f && q[0].h * q[4].h > 0.5f * m2)) atomicOr(flag, kErrNonphysical);
}

// FP32 reconstruction and flux with the FP64 update (GKS_PREC_MIXED_FP64UPD): the face sums
// accumulate the FP32 face fluxes in FP64, and the update reads and writes the FP64 state
// [5][nc], which is the master copy in this mode; the gather copies the reconstruction reads
// (float pairs) are written from it: Q* by stage 1, Q^{n+1} by stage 2.
template <bool kSecond>
__global__ void __launch_bounds__(256) k_stage_fd(
    int64_t nc, const int32_t* __restrict__ cf_ptr, const int32_t* __restrict__ cf_idx,
    const float* __restrict__ fface, const double* __restrict__ ivol, double c1, double c2,
    double* __restrict__ L, double* __restrict__ Lt, double* __restrict__ Q,
    float* __restrict__ QA, float* __restrict__ QsA, int* flag) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nc) return;
  double s[10];
#pragma unroll
  for (int q = 0; q < 10; ++q) s[q] = 0.0;
  for (int k = cf_ptr[i]; k < cf_ptr[i + 1]; ++k) {
    const int32_t e = __ldg(cf_idx + k);
    const float4* fp = reinterpret_cast<const float4*>(fface + (int64_t)kFaceStride * (e >> 1));
    const float4 a = __ldg(fp), b = __ldg(fp + 1), c = __ldg(fp + 2);
    const float x[10] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y};
    const double sg = (e & 1) ? 1.0 : -1.0;
#pragma unroll
    for (int q = 0; q < 10; ++q) s[q] += sg * (double)x[q];
  }
  const double iv = ivol[i];
  double q[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    const double qn = Q[v * nc + i];
    const double lt = s[5 + v] * iv;
    if (!kSecond) {
      const double l = s[v] * iv;
      L[v * nc + i] = l;
      Lt[v * nc + i] = lt;
      q[v] = qn + c1 * l + c2 * lt;
    } else {
      q[v] = qn + c1 * L[v * nc + i] + c2 * (Lt[v * nc + i] + 2.0 * lt);
      Q[v * nc + i] = q[v];
    }
  }
  Gq<float>::store(kSecond ? QA : QsA, i, q);
  if (!physical(q)) atomicOr(flag, kErrNonphysical);
}

template <bool kSecond>
__global__ void __launch_bounds__(256) k_stage_d(
    int64_t nc, const int32_t* __restrict__ cf_ptr, const int32_t* __restrict__ cf_idx,
    const double* __restrict__ fface, const double* __restrict__ ivol, double c1, double c2,
    double* __restrict__ L, double* __restrict__ Lt, double* __restrict__ QA,
    double* __restrict__ QsA, int* flag) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nc) return;
  double s[10];
  face_sums<double>(cf_ptr[i], cf_ptr[i + 1], cf_idx, fface, s);
  const double iv = ivol[i];
  Gq<double> g;
  g.load(QA, i);
  double q[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    const double lt = s[5 + v] * iv;
    if (!kSecond) {
      const double l = s[v] * iv;
      L[v * nc + i] = l;
      Lt[v * nc + i] = lt;
      q[v] = g.q[v] + c1 * l + c2 * lt;
    } else {
      q[v] = g.q[v] + c1 * L[v * nc + i] + c2 * (Lt[v * nc + i] + 2.0 * lt);
    }
  }
  Gq<double>::store(kSecond ? QA : QsA, i, q);
  if (!physical(q)) atomicOr(flag, kErrNonphysical);
}

// ------------------------------------------------------------------------------------------
// The two-stage combinations of Section 3.3 on caller arrays of n values, for a differentiable
// rollout built from residual calls: stage 1 out = Q + c1 L + c2 Lt (c1 = dt/2, c2 = dt^2/8),
// stage 2 out = Q + c1 L + c2 (Lt + 2 Lts) (c1 = dt, c2 = dt^2/6); and their transposes.
__global__ void __launch_bounds__(256) k_s2o4_stage(int64_t n, int stage, double c1, double c2,
                                                    const double* __restrict__ Q,
                                                    const double* __restrict__ L,
                                                    const double* __restrict__ Lt,
                                                    const double* __restrict__ Lts,
                                                    double* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double lt = stage == 1 ? Lt[i] : Lt[i] + 2.0 * Lts[i];
  out[i] = Q[i] + c1 * L[i] + c2 * lt;
}
__global__ void __launch_bounds__(256) k_s2o4_stage_vjp(int64_t n, int stage, double c1,
                                                        double c2, const double* __restrict__ g,
                                                        double* __restrict__ gQ,
                                                        double* __restrict__ gL,
                                                        double* __restrict__ gLt,
                                                        double* __restrict__ gLts) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double gi = g[i];
  gQ[i] = gi;
  gL[i] = c1 * gi;
  gLt[i] = c2 * gi;
  if (stage == 2) gLts[i] = 2.0 * c2 * gi;
}

// ------------------------------------------------------------------------------------------
// Implicit step (Section 4): backward Euler with the residual's change linearised by the flux
// splitting (T(Q_i) + T(Q_p) - r (Q_p - Q_i))/2 . n S, solved by Jacobi iterations:
//   (|Omega_i|/dt + 1/2 sum_f r_f S_f) dQ_i^(k)
//     = |Omega_i| Res_i - 1/2 sum_f [T_n(Q_p + dQ_p^(k-1)) - T_n(Q_p) - r_f dQ_p^(k-1)] S_f,
// |Omega_i| Res_i = s + dt/2 st (the face sums of F^n and dF/dt: the step-averaged GKS flux),
// r_f = max over the two sides of |U . n| + c at Q^n, n out of cell i; a wall face couples the
// cell to its mirror image. The Euler-flux change is formed from the increments themselves
// (du = (dm - u drho)/rho', dp = (gamma - 1)(dE - (m . du + dm . u')/2)), so no two nearly equal
// fluxes are subtracted.

template <class R>
__device__ __forceinline__ void state_of(const R* __restrict__ QA, int64_t c, R q[5]) {
  Gq<R> g;
  g.load(QA, c);
#pragma unroll
  for (int v = 0; v < 5; ++v) q[v] = (R)g.value(v);
}
template <class R>
__device__ __forceinline__ R wave_speed(const R q[5], const R n[3], R gm1) {
  const R ir = R(1) / q[0];
  const R u[3] = {q[1] * ir, q[2] * ir, q[3] * ir};
  const R p = gm1 * (q[4] - R(0.5) * (q[1] * u[0] + q[2] * u[1] + q[3] * u[2]));
  const R c2 = (gm1 + R(1)) * p * ir;
  return fabs(u[0] * n[0] + u[1] * n[1] + u[2] * n[2]) + sqrt(c2 > R(0) ? c2 : R(0));
}
template <class R>
__device__ __forceinline__ void euler_flux_change(const R q[5], const R d[5], const R n[3], R gm1,
                                                  R out[5]) {
  const R ir = R(1) / q[0], ir1 = R(1) / (q[0] + d[0]);
  R u[3], du[3], u1[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    u[a] = q[1 + a] * ir;
    du[a] = (d[1 + a] - u[a] * d[0]) * ir1;
    u1[a] = u[a] + du[a];
  }
  const R un = u[0] * n[0] + u[1] * n[1] + u[2] * n[2];
  const R dun = du[0] * n[0] + du[1] * n[1] + du[2] * n[2], un1 = un + dun;
  const R p = gm1 * (q[4] - R(0.5) * (q[1] * u[0] + q[2] * u[1] + q[3] * u[2]));
  const R dp = gm1 * (d[4] - R(0.5) * (q[1] * du[0] + q[2] * du[1] + q[3] * du[2] +
                                       d[1] * u1[0] + d[2] * u1[1] + d[3] * u1[2]));
  out[0] = d[1] * n[0] + d[2] * n[1] + d[3] * n[2];
#pragma unroll
  for (int a = 0; a < 3; ++a) out[1 + a] = d[1 + a] * un1 + q[1 + a] * dun + dp * n[a];
  out[4] = (d[4] + dp) * un1 + (q[4] + p) * dun;
}

// The wall's ghost of a cell state q and of an increment d of it: q_g = G(q), d_g = G(q + d) -
// G(q), with G the value part of wall_ghost. The slip and adiabatic maps are linear, so
// d_g = G(d); the isothermal map's energy row holds |m|^2 / rho, whose change is formed as
// (2 m . dm + |dm|^2 - |m|^2 drho / rho) / (rho + drho) without cancellation.
template <class R>
__device__ __forceinline__ void wall_cell_ghost(const FluxParams<R>& P, int code,
                                                const WallData<R>& wd, const R q[5], R qg[5]) {
  const R zg[5][3] = {};
  R gg[5][3];
  wall_ghost(P, code, wd, q, zg, qg, gg);
}
template <class R>
__device__ __forceinline__ void wall_cell_ghost_inc(const FluxParams<R>& P, int code,
                                                    const WallData<R>& wd, const R q[5],
                                                    const R d[5], R dg[5]) {
  const R zg[5][3] = {};
  R gg[5][3];
  if (code >= 12) {  // far field: the change of the characteristic state
    R q1[5], g0[5], g1[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) q1[v] = q[v] + d[v];
    wall_ghost(P, code, wd, q, zg, g0, gg);
    wall_ghost(P, code, wd, q1, zg, g1, gg);
#pragma unroll
    for (int v = 0; v < 5; ++v) dg[v] = g1[v] - g0[v];
    return;
  }
  if (code < 6 || wd.Tw <= R(0)) {
    wall_ghost(P, code, wd, d, zg, dg, gg);
    return;
  }
  const R u0 = wd.uw[0], u1 = wd.uw[1], u2 = wd.uw[2];
  const R uw2 = u0 * u0 + u1 * u1 + u2 * u2;
  dg[0] = d[0];
  dg[1] = R(2) * u0 * d[0] - d[1];
  dg[2] = R(2) * u1 * d[0] - d[2];
  dg[3] = R(2) * u2 * d[0] - d[3];
  const R mdm = q[1] * d[1] + q[2] * d[2] + q[3] * d[3];
  const R dm2 = d[1] * d[1] + d[2] * d[2] + d[3] * d[3];
  const R m2 = q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
  dg[4] = (R(2) * wd.Tw / (P.gamma - R(1)) + R(2) * uw2) * d[0] - d[4] +
          (R(2) * mdm + dm2 - m2 * d[0] / q[0]) / (q[0] + d[0]) -
          R(2) * (u0 * d[1] + u1 * d[2] + u2 * d[3]);
}

// The other side of cell-face entry e seen from cell i: its index (-1: the wall's ghost of cell
// i, *wall the wall code) and the unit normal out of cell i with the face area.
template <class R>
__device__ __forceinline__ int64_t other_side(int32_t e, const int32_t* __restrict__ f_owner,
                                              const int32_t* __restrict__ f_nb,
                                              const int8_t* __restrict__ f_wall,
                                              const R* __restrict__ fn, R n[3], R& S, int& wall) {
  const int64_t f = e >> 1;
  const bool nbside = e & 1;
  const R sg = nbside ? R(-1) : R(1);
#pragma unroll
  for (int a = 0; a < 3; ++a) n[a] = sg * fn[4 * f + a];
  S = fn[4 * f + 3];
  const int64_t p = nbside ? f_owner[f] : f_nb[f];
  wall = p < 0 ? f_wall[f] : -1;
  return p;
}

template <class R>
__global__ void __launch_bounds__(256) k_jacobi_init(
    int64_t nc, const int32_t* __restrict__ cf_ptr, const int32_t* __restrict__ cf_idx,
    const int32_t* __restrict__ f_owner, const int32_t* __restrict__ f_nb,
    const int8_t* __restrict__ f_wall, const R* __restrict__ fface, const R* __restrict__ fn,
    const double* __restrict__ vol, double dt, const R* __restrict__ QA, FluxParams<R> P,
    const R* __restrict__ wall_tab, R* __restrict__ Rv, R* __restrict__ D, R* __restrict__ hrs,
    R* __restrict__ dQ0) {
  const R gm1 = P.gamma - R(1);
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nc) return;
  R qi[5];
  state_of(QA, i, qi);
  R dsum = R(0);
  const int k0 = cf_ptr[i], k1 = cf_ptr[i + 1];
  for (int k = k0; k < k1; ++k) {
    R n[3], S, qp[5];
    int wall;
    const int64_t p = other_side(cf_idx[k], f_owner, f_nb, f_wall, fn, n, S, wall);
    if (p >= 0) {
      state_of(QA, p, qp);
    } else {
      wall_cell_ghost(P, wall, wall_data(wall_tab, wall), qi, qp);
    }
    const R r = fmax(wave_speed(qi, n, gm1), wave_speed(qp, n, gm1));
    hrs[k] = R(0.5) * r * S;
    dsum += hrs[k];
  }
  R res[5];
  if constexpr (std::is_same<R, float>::value) {
    ff s[10];
    face_sums_ff(k0, k1, cf_idx, fface, 0, s);
    const ff h = ff_from(0.5 * dt);
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const ff x = ff_add(s[v], ff_mul(h, s[5 + v]));
      res[v] = x.h + x.l;
    }
  } else {
    double s[10];
    face_sums<double>(k0, k1, cf_idx, fface, s);
#pragma unroll
    for (int v = 0; v < 5; ++v) res[v] = s[v] + 0.5 * dt * s[5 + v];
  }
  const R d = (R)(vol[i] / dt) + dsum;
  D[i] = d;
  const R id = R(1) / d;
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    Rv[v * nc + i] = res[v];
    dQ0[v * nc + i] = res[v] * id;
  }
}

template <class R, bool kLast>
__global__ void __launch_bounds__(256) k_jacobi_sweep(
    int64_t nc, const int32_t* __restrict__ cf_ptr, const int32_t* __restrict__ cf_idx,
    const int32_t* __restrict__ f_owner, const int32_t* __restrict__ f_nb,
    const int8_t* __restrict__ f_wall, const R* __restrict__ fn, const R* __restrict__ QA,
    const R* __restrict__ Rv, const R* __restrict__ D, const R* __restrict__ hrs,
    const R* __restrict__ dQin, R* __restrict__ dQout, R* __restrict__ QAout, FluxParams<R> P,
    const R* __restrict__ wall_tab, int* flag) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nc) return;
  const R gm1 = P.gamma - R(1);
  R acc[5] = {R(0), R(0), R(0), R(0), R(0)};
  const int k0 = cf_ptr[i], k1 = cf_ptr[i + 1];
  for (int k = k0; k < k1; ++k) {
    R n[3], S, qp[5], dp[5], dT[5];
    int wall;
    const int64_t p = other_side(cf_idx[k], f_owner, f_nb, f_wall, fn, n, S, wall);
    const int64_t c = p >= 0 ? p : i;
    state_of(QA, c, qp);
#pragma unroll
    for (int v = 0; v < 5; ++v) dp[v] = dQin[v * nc + c];
    if (p < 0) {  // the wall's ghost of the cell and of its increment
      R qg[5], dg[5];
      const WallData<R> wd = wall_data(wall_tab, wall);
      wall_cell_ghost(P, wall, wd, qp, qg);
      wall_cell_ghost_inc(P, wall, wd, qp, dp, dg);
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        qp[v] = qg[v];
        dp[v] = dg[v];
      }
    }
    euler_flux_change(qp, dp, n, gm1, dT);
    const R h = hrs[k];
#pragma unroll
    for (int v = 0; v < 5; ++v) acc[v] += R(0.5) * S * dT[v] - h * dp[v];
  }
  const R id = R(1) / D[i];
  R d[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) d[v] = (Rv[v * nc + i] - acc[v]) * id;
  if (!kLast) {
#pragma unroll
    for (int v = 0; v < 5; ++v) dQout[v * nc + i] = d[v];
    return;
  }
  // Q^{n+1} = Q^n + dQ, written to the other gather copy (neighbours still read Q^n)
  if constexpr (std::is_same<R, float>::value) {
    Gq<float> g;
    g.load(QA, i);
    ff q[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) q[v] = ff_add(ff{g.hi[v], g.lo[v]}, ff{d[v], 0.f});
    Gq<float>::store_ff(QAout, i, q);
    const float m2 = q[1].h * q[1].h + q[2].h * q[2].h + q[3].h * q[3].h;
    if (!(q[0].h > 0.f && q[0].h * q[4].h > 0.5f * m2)) atomicOr(flag, kErrNonphysical);
  } else {
    Gq<double> g;
    g.load(QA, i);
    double q[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) q[v] = g.q[v] + d[v];
    Gq<double>::store(QAout, i, q);
    if (!physical(q)) atomicOr(flag, kErrNonphysical);
  }
}

template <class R>
__global__ void k_unpack(int64_t nc, const R* __restrict__ QA, double* __restrict__ Q) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nc) return;
  Gq<R> g;
  g.load(QA, i);
#pragma unroll
  for (int v = 0; v < 5; ++v) Q[v * nc + i] = unpack_value(g, v);
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
  if (!physical(q)) atomicOr(flag, kErrNonphysical);
}

constexpr int kDtThreads = 256;
constexpr int kDtMaxBlocks = 1024;

__global__ void __launch_bounds__(kDtThreads) k_dt_partial(int64_t nc, const double* __restrict__ Q,
                                                           const double* __restrict__ hdt,
                                                           double gamma, double mu, int power,
                                                           double T_ref, double mu_pow,
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
    // viscosity at the cell's temperature p / rho (the power law of Section 5.4, else constant)
    const double mue = power ? mu * pow(p / (r * T_ref), mu_pow) : mu;
    const double bound = h / (sqrt(u2) + c + 2.0 * mue / (r * h));
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

// Largest dynamic shared memory of one block (227 KB on this architecture).
constexpr size_t kMaxBlockSmem = 227 * 1024;

// Shared memory of one SM and the part the hardware keeps for each resident block.
constexpr size_t kSmemPerSM = 228 * 1024, kSmemPerBlockReserved = 1024;

inline int recon_blocks_per_sm(size_t smem) {
  return (int)(kSmemPerSM / (smem + kSmemPerBlockReserved));
}

template <class R, bool kPf, bool kStB>
void launch_recon_range(const DevMesh& m, const GeoR<R>& g, const KParams<R>& p, const R* QA,
                        R* poly, int* flag, int r, size_t smem, cudaStream_t st) {
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_recon<R, kPf, kStB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
  ReconUni u{m.rr.uni[r], m.rr.K[r], m.rr.S[r], m.rr.cnt[r], m.rr.st0[r], m.rr.sb0[r]};
  k_recon<R, kPf, kStB><<<(unsigned)(m.rr.t1[r] - m.rr.t0[r]), kReconThreads, smem, st>>>(
      m.nc, m.rr.t0[r], m.rr.K[r], m.rr.S[r], m.rr.M[r], u, QA, m.t_K, m.t_cnt, m.t_st, m.t_sb,
      m.t_idx, m.n_sub, g.Ap, g.Bp, g.mom, g.h, p.weno_gamma, p.weno_eps, p.weno_pow, poly, flag,
      p.wait_tries, p.withhold);
}

// Ghost slots of moving no-slip walls and far-field planes: QA[nc + g] = the image's flow
// variables from QA[g_src[g]]. Linear slots apply their composed map; the others apply the
// maps of their planes in order (slip: normal momentum negated; no-slip: rho kept,
// m -> 2 U_w rho - m, E -> E + 2 |U_w|^2 rho - 2 U_w . m; far field: the characteristic
// state), in precision R.
template <class R>
__global__ void __launch_bounds__(128) k_ghost_fill(int64_t nc, int64_t ng,
                                                    const int32_t* __restrict__ src,
                                                    const double* __restrict__ map,
                                                    const float* __restrict__ mapf,
                                                    const uint8_t* __restrict__ chain, int bcs,
                                                    FluxParams<R> P, const R* __restrict__ wall_tab,
                                                    R* QA) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= ng) return;
  Gq<R> g;
  g.load(QA, src[k]);
  if (const int code = chain[k]) {
    R q[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) q[v] = (R)g.value(v);
    for (int s = 0; s < 2; ++s) {
      const int w = ((code >> (3 * s)) & 7) - 1;
      if (w < 0) break;
      const int ax = w % 3, kind = (bcs >> (2 * ax)) & 3;
      if (kind == 1) {
        q[1 + ax] = -q[1 + ax];
      } else if (kind == 2) {
        const R* t = wall_tab + kPlaneStride * w;
        const R um = t[0] * q[1] + t[1] * q[2] + t[2] * q[3];
        q[4] = q[4] + R(2) * (t[0] * t[0] + t[1] * t[1] + t[2] * t[2]) * q[0] - R(2) * um;
#pragma unroll
        for (int a = 0; a < 3; ++a) q[1 + a] = R(2) * t[a] * q[0] - q[1 + a];
      } else {
        R o[5];
        farfield_state(P, wall_tab + kPlaneStride * w + 4, ax, w >= 3 ? R(1) : R(-1), q, o);
#pragma unroll
        for (int v = 0; v < 5; ++v) q[v] = o[v];
      }
    }
    if constexpr (std::is_same<R, float>::value) {
      ff o[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) o[v] = ff{q[v], 0.f};
      Gq<float>::store_ff(QA, nc + k, o);
    } else {
      Gq<double>::store(QA, nc + k, q);
    }
    return;
  }
  if constexpr (std::is_same<R, float>::value) {
    const float* c = mapf + 20 * k;
    auto co = [&](int j) { return ff{c[2 * j], c[2 * j + 1]}; };
    ff q[5], o[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) q[v] = ff{g.hi[v], g.lo[v]};
    o[0] = q[0];
    o[4] = ff_add(q[4], ff_mul(co(6), q[0]));
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const float sj = c[2 * j];  // +-1, exact
      o[1 + j] = ff_add(ff{sj * q[1 + j].h, sj * q[1 + j].l}, ff_mul(co(3 + j), q[0]));
      o[4] = ff_add(o[4], ff_mul(co(7 + j), q[1 + j]));
    }
    Gq<float>::store_ff(QA, nc + k, o);
  } else {
    const double* c = map + 10 * k;
    double o[5];
    o[0] = g.q[0];
    o[4] = g.q[4] + c[6] * g.q[0];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      o[1 + j] = c[j] * g.q[1 + j] + c[3 + j] * g.q[0];
      o[4] += c[7 + j] * g.q[1 + j];
    }
    Gq<double>::store(QA, nc + k, o);
  }
}

// One launch per tile range, the bulk-copy variant whenever its shared memory fits a block. The
// ranges are independent: with fj, range r > 0 runs on auxiliary stream r - 1, forked from and
// joined back into st, so that the ranges' blocks share the GPU.
template <class R>
void launch_recon(const DevMesh& m, const GeoR<R>& g, const KParams<R>& p, const R* QA,
                  R* poly, int* flag, cudaStream_t st, const ForkJoin* fj) {
  // the ghost slots beyond nc belong to the reconstruction: refresh them from the state first
  if (m.ng > 0)
    k_ghost_fill<R><<<blocks_for(m.ng, 128), 128, 0, st>>>(
        m.nc, m.ng, m.g_src, m.g_map, m.g_mapf, m.g_chain, m.bcs, flux_params(p),
        wall_table<R>(m), const_cast<R*>(QA));
  int used = 0;
  const bool fork = fj && fj->n > 0 && m.rr.n > 1;
  if (fork) cudaEventRecord(fj->fork, st);
  for (int r = 0; r < m.rr.n; ++r) {
    if (m.rr.t1[r] <= m.rr.t0[r]) continue;
    cudaStream_t s = st;
    if (fork && r > 0 && used < fj->n) {
      s = fj->aux[used];
      cudaStreamWaitEvent(s, fj->fork, 0);
    }
    // the sub-stencil entries are staged in shared memory only where that costs the range no
    // resident blocks below the register bound; otherwise they are prefetched into L2 like the
    // rows (on the 64^3-cube mesh the pyramid and hexahedron ranges: 3 and 4 blocks per SM with
    // the entries staged, 5 without; 0.595 -> 0.571 ms per FP32 pass)
    const ReconSmem<R> pb(m.rr.K[r], m.rr.S[r], m.rr.M[r], true, true);
    const ReconSmem<R> pl(m.rr.K[r], m.rr.S[r], m.rr.M[r], true, false);
    const int nb_l = std::min(kReconBlocksPerSM, recon_blocks_per_sm(pl.bytes));
    if (pb.bytes <= kMaxBlockSmem && recon_blocks_per_sm(pb.bytes) >= nb_l) {
      launch_recon_range<R, true, true>(m, g, p, QA, poly, flag, r, pb.bytes, s);
    } else if (pl.bytes <= kMaxBlockSmem) {
      launch_recon_range<R, true, false>(m, g, p, QA, poly, flag, r, pl.bytes, s);
    } else {
      const ReconSmem<R> np(m.rr.K[r], m.rr.S[r], m.rr.M[r], false, false);
      launch_recon_range<R, false, false>(m, g, p, QA, poly, flag, r, np.bytes, s);
    }
    if (s != st) {
      cudaEventRecord(fj->join[used], s);
      cudaStreamWaitEvent(st, fj->join[used], 0);
      ++used;
    }
  }
}
template <class R>
void launch_flux(const DevMesh& m, const GeoR<R>& g, const KParams<R>& p, const R* poly,
                 const R* QA, double dt, R* fface, int* flag, cudaStream_t st) {
  const FluxParams<R> fp = flux_params(p);
  const unsigned nb = blocks_for(4 * m.nf, 128);
  auto kern = fp.full ? (fp.tau_model == 0 ? k_flux<R, true, true> : k_flux<R, true, false>)
                      : (fp.tau_model == 0 ? k_flux<R, false, true> : k_flux<R, false, false>);
  kern<<<nb, 128, 0, st>>>(m.nf, m.nc, m.f_owner, m.f_nb, m.f_wall, g.fgp, poly, QA,
                           p.gp_fallback, fp, wall_table<R>(m), (R)dt, fface, flag);
}
template <class R>
void launch_gather(const DevMesh& m, const Geo64& g, const R* fface, double* L, double* Lt,
                   cudaStream_t st) {
  k_gather<R><<<blocks_for(m.nc, 256), 256, 0, st>>>(m.nc, m.cf_ptr, m.cf_idx, fface, g.ivol, L,
                                                       Lt);
}
template <class R>
void launch_stage(const DevMesh& m, const GeoR<R>& g, const R* fface, int stage, double dt,
                  void* L, void* Lt, R* QA, R* QsA, int* flag, cudaStream_t st, double* Q64,
                  const double* ivol64) {
  const unsigned nb = blocks_for(m.nc, 256);
  // stage 1: c1 = dt/2, c2 = dt^2/8; stage 2: c1 = dt, c2 = dt^2/6
  const double c1 = stage == 1 ? 0.5 * dt : dt, c2 = stage == 1 ? dt * dt / 8.0 : dt * dt / 6.0;
  if constexpr (std::is_same<R, float>::value) {
    if (Q64) {  // FP64 update of the FP64 master state
      double* l = static_cast<double*>(L);
      double* lt = static_cast<double*>(Lt);
      if (stage == 1)
        k_stage_fd<false><<<nb, 256, 0, st>>>(m.nc, m.cf_ptr, m.cf_idx, fface, ivol64, c1, c2, l,
                                              lt, Q64, QA, QsA, flag);
      else
        k_stage_fd<true><<<nb, 256, 0, st>>>(m.nc, m.cf_ptr, m.cf_idx, fface, ivol64, c1, c2, l,
                                             lt, Q64, QA, QsA, flag);
      return;
    }
    ff* l = static_cast<ff*>(L);
    ff* lt = static_cast<ff*>(Lt);
    const ff* iv = reinterpret_cast<const ff*>(g.ivol);
    if (stage == 1)
      k_stage_f<false><<<nb, 256, 0, st>>>(m.nc, m.cf_ptr, m.cf_idx, fface, iv, ff_from(c1),
                                           ff_from(c2), l, lt, QA, QsA, flag);
    else
      k_stage_f<true><<<nb, 256, 0, st>>>(m.nc, m.cf_ptr, m.cf_idx, fface, iv, ff_from(c1),
                                          ff_from(c2), l, lt, QA, QsA, flag);
  } else {
    double* l = static_cast<double*>(L);
    double* lt = static_cast<double*>(Lt);
    if (stage == 1)
      k_stage_d<false><<<nb, 256, 0, st>>>(m.nc, m.cf_ptr, m.cf_idx, fface, g.ivol, c1, c2, l, lt,
                                           QA, QsA, flag);
    else
      k_stage_d<true><<<nb, 256, 0, st>>>(m.nc, m.cf_ptr, m.cf_idx, fface, g.ivol, c1, c2, l, lt,
                                          QA, QsA, flag);
  }
}
void launch_s2o4_stage(int64_t n, int stage, double dt, const double* Q, const double* L,
                       const double* Lt, const double* Lts, double* out, cudaStream_t st) {
  const double c1 = stage == 1 ? 0.5 * dt : dt, c2 = stage == 1 ? dt * dt / 8.0 : dt * dt / 6.0;
  k_s2o4_stage<<<blocks_for(n, 256), 256, 0, st>>>(n, stage, c1, c2, Q, L, Lt, Lts, out);
}
void launch_s2o4_stage_vjp(int64_t n, int stage, double dt, const double* g, double* gQ,
                           double* gL, double* gLt, double* gLts, cudaStream_t st) {
  const double c1 = stage == 1 ? 0.5 * dt : dt, c2 = stage == 1 ? dt * dt / 8.0 : dt * dt / 6.0;
  k_s2o4_stage_vjp<<<blocks_for(n, 256), 256, 0, st>>>(n, stage, c1, c2, g, gQ, gL, gLt, gLts);
}

template <class R>
void launch_jacobi_init(const DevMesh& m, const R* fface, const R* fn, const double* vol,
                        double dt, const R* QA, R* Rv, R* D, R* hrs, R* dQ0,
                        const KParams<R>& kp, cudaStream_t st) {
  k_jacobi_init<R><<<blocks_for(m.nc, 256), 256, 0, st>>>(m.nc, m.cf_ptr, m.cf_idx, m.f_owner,
                                                          m.f_nb, m.f_wall, fface, fn, vol, dt,
                                                          QA, flux_params(kp), wall_table<R>(m),
                                                          Rv, D, hrs, dQ0);
}
template <class R>
void launch_jacobi_sweep(const DevMesh& m, const R* fn, const R* QA, const R* Rv, const R* D,
                         const R* hrs, const R* dQin, R* dQout, int last, R* QAout,
                         const KParams<R>& kp, int* flag, cudaStream_t st) {
  const unsigned nb = blocks_for(m.nc, 256);
  const FluxParams<R> fp = flux_params(kp);
  if (last)
    k_jacobi_sweep<R, true><<<nb, 256, 0, st>>>(m.nc, m.cf_ptr, m.cf_idx, m.f_owner, m.f_nb,
                                                m.f_wall, fn, QA, Rv, D, hrs, dQin, dQout, QAout,
                                                fp, wall_table<R>(m), flag);
  else
    k_jacobi_sweep<R, false><<<nb, 256, 0, st>>>(m.nc, m.cf_ptr, m.cf_idx, m.f_owner, m.f_nb,
                                                 m.f_wall, fn, QA, Rv, D, hrs, dQin, dQout, QAout,
                                                 fp, wall_table<R>(m), flag);
}
template <class R>
void launch_unpack(int64_t nc, const R* QA, double* Q, cudaStream_t st) {
  k_unpack<R><<<blocks_for(nc, 256), 256, 0, st>>>(nc, QA, Q);
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
void launch_dt(int64_t nc, const double* Q, const double* hdt, double gamma, double mu, int power,
               double T_ref, double mu_pow, double* partial, int nblocks, double* out,
               cudaStream_t st) {
  k_dt_partial<<<nblocks, kDtThreads, 0, st>>>(nc, Q, hdt, gamma, mu, power, T_ref, mu_pow,
                                               partial);
  k_dt_final<<<1, 256, 0, st>>>(partial, nblocks, out);
}

template void launch_recon<double>(const DevMesh&, const GeoR<double>&, const KParams<double>&,
                                   const double*, double*, int*, cudaStream_t, const ForkJoin*);
template void launch_permute_in<double>(int64_t, const int32_t*, const double*, double*, double*,
                                        cudaStream_t);
template void launch_permute_in<float>(int64_t, const int32_t*, const double*, double*, float*,
                                       cudaStream_t);
template void launch_recon<float>(const DevMesh&, const GeoR<float>&, const KParams<float>&,
                                  const float*, float*, int*, cudaStream_t, const ForkJoin*);
template void launch_flux<double>(const DevMesh&, const GeoR<double>&, const KParams<double>&,
                                  const double*, const double*, double, double*, int*,
                                  cudaStream_t);
template void launch_flux<float>(const DevMesh&, const GeoR<float>&, const KParams<float>&,
                                 const float*, const float*, double, float*, int*, cudaStream_t);
template void launch_gather<double>(const DevMesh&, const Geo64&, const double*, double*, double*,
                                    cudaStream_t);
template void launch_gather<float>(const DevMesh&, const Geo64&, const float*, double*, double*,
                                   cudaStream_t);
template void launch_stage<double>(const DevMesh&, const GeoR<double>&, const double*, int, double,
                                   void*, void*, double*, double*, int*, cudaStream_t, double*,
                                   const double*);
template void launch_stage<float>(const DevMesh&, const GeoR<float>&, const float*, int, double,
                                  void*, void*, float*, float*, int*, cudaStream_t, double*,
                                  const double*);
template void launch_unpack<double>(int64_t, const double*, double*, cudaStream_t);
template void launch_jacobi_init<double>(const DevMesh&, const double*, const double*,
                                         const double*, double, const double*, double*, double*,
                                         double*, double*, const KParams<double>&, cudaStream_t);
template void launch_jacobi_init<float>(const DevMesh&, const float*, const float*, const double*,
                                        double, const float*, float*, float*, float*, float*,
                                        const KParams<float>&, cudaStream_t);
template void launch_jacobi_sweep<double>(const DevMesh&, const double*, const double*,
                                          const double*, const double*, const double*,
                                          const double*, double*, int, double*,
                                          const KParams<double>&, int*, cudaStream_t);
template void launch_jacobi_sweep<float>(const DevMesh&, const float*, const float*, const float*,
                                         const float*, const float*, const float*, float*, int,
                                         float*, const KParams<float>&, int*, cudaStream_t);
template void launch_unpack<float>(int64_t, const float*, double*, cudaStream_t);

}  // namespace gks

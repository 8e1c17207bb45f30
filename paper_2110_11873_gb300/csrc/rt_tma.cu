// The FP32 operator apply of single problems (sm_103a): a vectorised
// quadrature (J, Eq. 11-14) that also forms the multipolar components
// (Eq. 13-14), and a formal solver (Eq. 9-10) whose input streams through
// shared memory with tensor copies.
//
//   k_quad     partial moments.  Each thread owns four consecutive rays (one
//              16-byte load per Stokes parameter and height) and keeps their
//              quadrature weights in registers:  w0 = w_m w_p,
//              w1 = w0 T201_m, w2 = w0 T202_m, so that
//              J00_k = sum_r w0 x_I  and  J20_k = sum_r (w1 x_I + w2 x_Q).
//              A CTA covers 1024 rays and a range of heights; warp sums are
//              combined in a fixed order into one partial per (height, CTA
//              column).  The last CTA of a grid row to finish (a counter per
//              row) sums that row's partials over the columns in column order
//              and writes sigma00 = xi J00, sigma20 = xi W2 J20 (with the
//              local-Lambda block inverse in that mode) into the operand
//              tables of the formal solver.  Which CTA finishes last does not
//              change the sums, so the result does not depend on scheduling.
//              k_quad_norm is the same inside GMRES with FP64 basis vectors:
//              it also ends the previous Arnoldi step and forms its input
//              v = u / ||u|| as it reads u.
//   k_staged   the formal solve (a programmatic dependent of the quadrature:
//              its set-up, and in a standalone apply its first tensor copies
//              of x, overlap the quadrature's tail).  A CTA takes 32 rays of
//              one direction sign and splits the depth into `ntile` tiles,
//              one warp each; the depth recurrence
//              I_k = e I_prev + alpha S_prev + beta S_k is solved as an affine
//              scan (tile maps, chained inflows, re-sweep).  The step
//              coefficients are recomputed in FP32 from the node table and
//              the ray's scale; where Delta is small, alpha and beta come from
//              one Taylor series.  In the re-sweep every warp streams its rows of x (and
//              of the Jacobi diagonal) into a ring of shared-memory stages
//              with cp.async.bulk.tensor, one 3D box (rays x heights x Stokes)
//              per stage completing on an mbarrier, so the recurrence never
//              waits on HBM.  The per-node operands (sigma00, sigma20 and the
//              interval's optical depth) come from a table indexed along the
//              march, so both directions read it forwards; S_I and S_Q follow
//              from the lane's T201_m, T202_m (Eq. 7-8).
//
// Every mbarrier wait is bounded (kWaitNs of wall time): a warp whose copy
// does not arrive sets the problem's device error flag, waits (again
// bounded) for its copies still in flight and returns.
//
// Used when the tensor-copy and vector-load alignment rules hold (x 16-byte
// aligned, Nmu*Nnu and Nmu/2*Nnu multiples of 4); otherwise the
// register-ring kernels of rt_operator.cu run.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "rt_device.cuh"

namespace rt {

namespace {

#ifndef RT_STAGED_DK
#define RT_STAGED_DK 8
#endif
#ifndef RT_STAGED_NST
#define RT_STAGED_NST 2
#endif
#ifndef RT_STAGED_RS
#define RT_STAGED_RS 2
#endif
#ifndef RT_STAGED_MAXT
#define RT_STAGED_MAXT 16
#endif
#ifndef RT_STAGED_MINB
#define RT_STAGED_MINB 2
#endif

constexpr int kNST = RT_STAGED_NST;            // stages per warp
constexpr int kRS = RT_STAGED_RS;              // prefetch distance of the node operands (steps)
constexpr int kMaxT = RT_STAGED_MAXT;          // warps per CTA (depth tiles of a ray group)
constexpr int kTabPad = 2 * kRS;               // table entries past the last node (prefetch reads them)
constexpr unsigned long long kWaitNs = 1000000000ull;   // bound of one wait
constexpr int kQuadThreads = 256;
constexpr int kQuadMaxHeights = 64;            // heights per CTA of k_quad
constexpr int kQuadBatch = 2;                  // heights per batch of loads (two batches in flight)
constexpr int kQuadFinal = 4096;               // partials a row's last CTA stages in shared memory

template <typename TV, int MODE>
struct Cfg {
  // depth steps per stage: FP64 vectors use half the steps of FP32 ones
  static constexpr int DK = sizeof(TV) == 4 ? RT_STAGED_DK : RT_STAGED_DK / 2;
  static constexpr bool JAC = MODE == KM_JACOBI;
  static constexpr int XBYTES = 2 * DK * 32 * (int)sizeof(TV);   // x box
  static constexpr int DBYTES = JAC ? 2 * DK * 32 * 8 : 0;       // Jacobi diagonal box
  static constexpr int STAGE = XBYTES + DBYTES;
  static constexpr int WARP = kNST * STAGE + kNST * 8;           // stages and their barriers
  static_assert(DK % kRS == 0, "the operand ring divides a stage");
  static_assert(XBYTES % 128 == 0 && STAGE % 128 == 0, "tensor-copy destinations stay 128-byte aligned");
};

// Dynamic shared memory of a CTA of ntile warps: the stages of all warps
// (each a multiple of 128 bytes, from a 128-byte aligned base), then the
// barriers of all warps.
constexpr size_t smem_bytes(int warp_bytes, int ntile) { return 128 + (size_t)ntile * warp_bytes; }
static_assert(smem_bytes(Cfg<double, KM_JACOBI>::WARP, kMaxT) <= 227 * 1024, "a CTA fits the shared memory");

// ------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// wait for the phase of `parity` to complete; false after kWaitNs
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = gtimer();
  while (!mbar_try_wait(bar, parity))
    if (gtimer() - t0 > kWaitNs) return false;
  return true;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* tm, int c0, int c1, int c2,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void prefetch_tensormap(const CUtensorMap* tm) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(tm)) : "memory");
}

// 2^a by the hardware's approximate exponential (a <= 0 here)
__device__ __forceinline__ float ex2_approx(float a) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
  return r;
}

// ------------------------------------------------------ step coefficients
// The coefficients of I_k = e I_prev + alpha S_prev + beta S_k from the node
// operand op (op.z, op.w: the interval constants of the table) and the ray's
// scale rsc = phi_hat_p / |mu_m| (irsc = 1 / rsc); Delta = dtau * rsc.
//   DELO-linear: op.z = dtau / ln 2, op.w = 1 / dtau; D2 = Delta / ln 2 and
//     e = 2^(-D2) = exp(-Delta).  With q = (1 - e) / Delta, beta = 1 - q and
//     alpha = q - e.  For Delta < 1/2 those differences cancel, so there
//       h = beta / Delta = sum_n (-Delta)^n / (n+2)!   (from the series of
//       e^-Delta), truncated after n = 7 (relative error below 1e-8),
//       beta = Delta h,   alpha = Delta (1 - (1 + Delta) h),
//     the last from 1 - e = Delta g, g = 1 - Delta h, alpha = (1 - e) - beta;
//     1 - (1 + Delta) h stays near 1/2, so alpha keeps its relative accuracy.
//     Both branches are evaluated and one is selected (no divergence).
//     Above 1/2, q's rounding error is below 2e-7.
//   implicit Euler: op.z = dtau; e = 1 / (1 + Delta), alpha = 0, beta = Delta e.
//   trapezoidal: op.z = dtau; h = Delta / 2, q = 1 / (1 + h), e = (1 - h) q,
//     alpha = beta = h q.
//   (reciprocals by the hardware approximation, within 2 ulp)
constexpr double kLn2 = 0.69314718055994530942;
constexpr float kSeriesD2 = (float)(0.5 / kLn2);

// (-1)^n ln2^(n+1) / (n+2)!: the series of beta / D2 in powers of D2
constexpr double pow_ln2(int k) { return k == 0 ? 1.0 : kLn2 * pow_ln2(k - 1); }
constexpr double fact(int k) { return k <= 1 ? 1.0 : k * fact(k - 1); }
constexpr float kB(int n) { return (float)((n % 2 ? -1.0 : 1.0) * pow_ln2(n + 1) / fact(n + 2)); }

template <int FS>
__device__ __forceinline__ void step_coeffs(const float4& op, float rsc, float irsc, float& e, float& al, float& be) {
  if (FS == RT_FS_DELO_LINEAR) {
    const float D2 = op.z * rsc;
    e = ex2_approx(-D2);
    float hb = kB(7);
    hb = fmaf(hb, D2, kB(6));
    hb = fmaf(hb, D2, kB(5));
    hb = fmaf(hb, D2, kB(4));
    hb = fmaf(hb, D2, kB(3));
    hb = fmaf(hb, D2, kB(2));
    hb = fmaf(hb, D2, kB(1));
    hb = fmaf(hb, D2, kB(0));
    const float bs = hb * D2;
    const float onep = fmaf(D2, (float)kLn2, 1.0f);
    const float as = D2 * fmaf(-onep, hb, (float)kLn2);
    const float iD = op.w * irsc;
    const float q = fmaf(-e, iD, iD);
    const bool thin = D2 < kSeriesD2;
    be = thin ? bs : 1.0f - q;
    al = thin ? as : q - e;
  } else if (FS == RT_FS_IMPLICIT_EULER) {
    const float D = op.z * rsc;
    e = __fdividef(1.0f, 1.0f + D);
    al = 0.0f;
    be = D * e;
  } else {
    const float h = 0.5f * op.z * rsc;
    const float q = __fdividef(1.0f, 1.0f + h);
    e = (1.0f - h) * q;
    al = h * q;
    be = al;
  }
}

// ---------------------------------------------------------------- k_quad
template <typename TV>
__device__ __forceinline__ float4 load4(const TV* p);
template <>
__device__ __forceinline__ float4 load4<float>(const float* p) {
  return __ldg(reinterpret_cast<const float4*>(p));
}
template <>
__device__ __forceinline__ float4 load4<double>(const double* p) {
  const double2 a = __ldg(reinterpret_cast<const double2*>(p)), b = __ldg(reinterpret_cast<const double2*>(p) + 1);
  return make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
}

// four FP64 values of u scaled by inv: stored to xo (the GMRES normalisation
// v = u / ||u||) and returned in FP32 for the quadrature
__device__ __forceinline__ float4 load4_scaled(const double* u, double inv, double* xo) {
  double2 a = __ldg(reinterpret_cast<const double2*>(u)), b = __ldg(reinterpret_cast<const double2*>(u) + 1);
  a.x *= inv;
  a.y *= inv;
  b.x *= inv;
  b.y *= inv;
  reinterpret_cast<double2*>(xo)[0] = a;
  reinterpret_cast<double2*>(xo)[1] = b;
  return make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
}

// Where the quadrature puts its result: the multipolar components of every
// height go into the .xy of the formal solver's node tables, march-indexed
// per direction (tab[k] downward, tab[Ns + kTabPad + Ns-1-k] upward).
struct QuadOut {
  float* part;          // [Ns][gridDim.x][2] partial moments
  int* cnt;             // [rows] CTAs of a grid row done (reset by the last one)
  float4* tab;          // [2][Ns + kTabPad] node operands
  const double* Minv;   // [Ns][4] local-Lambda block inverses (KM_LOCAL_LAMBDA)
  float xi, xiW2;
  int Ns;
};

// Transposing warp sum of four FP32 values (7 shuffles and additions a lane
// instead of 20): lanes 0, 8, 16 and 24 end with the warp sums of v[0],
// v[1], v[2] and v[3]; fixed order.
__device__ __forceinline__ float warp_sum4f(const float* v) {
  const int lane = threadIdx.x & 31;
  const bool h16 = lane & 16, h8 = lane & 8;
  const float r0 = (h16 ? v[2] : v[0]) + __shfl_xor_sync(0xffffffffu, h16 ? v[0] : v[2], 16);
  const float r1 = (h16 ? v[3] : v[1]) + __shfl_xor_sync(0xffffffffu, h16 ? v[1] : v[3], 16);
  float t = (h8 ? r1 : r0) + __shfl_xor_sync(0xffffffffu, h8 ? r0 : r1, 8);
  t += __shfl_xor_sync(0xffffffffu, t, 4);
  t += __shfl_xor_sync(0xffffffffu, t, 2);
  t += __shfl_xor_sync(0xffffffffu, t, 1);
  return t;
}

// The partials of the heights of row ky of the grid, rays of column
// blockIdx.x (all threads of the CTA call it); the last CTA of the row then
// forms sigma00, sigma20 of the row's heights.  Loads run one batch of
// kQuadBatch heights ahead of the sums, so the memory system always has
// this CTA's next rows in flight.  NORM: the input is u * inv, written to xo
// as it is read.
template <typename TV, int MODE, bool NORM>
__device__ __forceinline__ void quad_tile(const TV* __restrict__ x, const double* __restrict__ dinv,
                                          const float* __restrict__ qw, int64_t nray, int hpc, const QuadOut& Q,
                                          int ky, const double* __restrict__ u = nullptr, double inv = 1.0,
                                          double* __restrict__ xo = nullptr) {
  constexpr int nw = kQuadThreads / 32;
  constexpr int U = kQuadBatch;
  static_assert(U == 2, "the transposing reduction takes two heights of two values");
  __shared__ float red[kQuadMaxHeights][nw][2];
  __shared__ float fin[kQuadFinal];
  __shared__ int last;
  const int Ns = Q.Ns;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t nc = nray / 4;
  const int64_t c = (int64_t)blockIdx.x * kQuadThreads + threadIdx.x;
  const bool ok = c < nc;
  const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 w0 = ok ? __ldg(reinterpret_cast<const float4*>(qw) + c) : z;
  const float4 w1 = ok ? __ldg(reinterpret_cast<const float4*>(qw + nray) + c) : z;
  const float4 w2 = ok ? __ldg(reinterpret_cast<const float4*>(qw + 2 * nray) + c) : z;
  const int k_lo = ky * hpc, k_hi = min(Ns, k_lo + hpc);
  const int64_t plane = (int64_t)Ns * nray;
  auto load = [&](int k, float4* vI, float4* vQ) {
#pragma unroll
    for (int v = 0; v < U; ++v) {
      vI[v] = z;
      vQ[v] = z;
      if (ok && k + v < k_hi) {
        const int64_t o = (int64_t)(k + v) * nray + 4 * c;
        if (NORM) {
          vI[v] = load4_scaled(u + o, inv, xo + o);
          vQ[v] = load4_scaled(u + plane + o, inv, xo + plane + o);
        } else {
          vI[v] = load4<TV>(x + o);
          vQ[v] = load4<TV>(x + plane + o);
        }
        if (MODE == KM_JACOBI) {
          const float4 dI = load4<double>(dinv + o), dQ = load4<double>(dinv + plane + o);
          vI[v] = make_float4(vI[v].x * dI.x, vI[v].y * dI.y, vI[v].z * dI.z, vI[v].w * dI.w);
          vQ[v] = make_float4(vQ[v].x * dQ.x, vQ[v].y * dQ.y, vQ[v].z * dQ.z, vQ[v].w * dQ.w);
        }
      }
    }
  };
  auto reduce = [&](int k, const float4* vI, const float4* vQ) {
    float a[2 * U];
#pragma unroll
    for (int v = 0; v < U; ++v) {
      float a0 = w0.x * vI[v].x;
      a0 = fmaf(w0.y, vI[v].y, a0);
      a0 = fmaf(w0.z, vI[v].z, a0);
      a0 = fmaf(w0.w, vI[v].w, a0);
      float a2 = w1.x * vI[v].x;
      a2 = fmaf(w1.y, vI[v].y, a2);
      a2 = fmaf(w1.z, vI[v].z, a2);
      a2 = fmaf(w1.w, vI[v].w, a2);
      a2 = fmaf(w2.x, vQ[v].x, a2);
      a2 = fmaf(w2.y, vQ[v].y, a2);
      a2 = fmaf(w2.z, vQ[v].z, a2);
      a2 = fmaf(w2.w, vQ[v].w, a2);
      a[2 * v] = a0;
      a[2 * v + 1] = a2;
    }
    const float t = warp_sum4f(a);   // lane 8*i holds the sum of a[i]
    if ((lane & 7) == 0) {
      const int i = lane >> 3, v = i >> 1;
      if (k + v < k_hi) red[k + v - k_lo][warp][i & 1] = t;
    }
  };
  float4 aI[U], aQ[U], bI[U], bQ[U];
  load(k_lo, aI, aQ);
  for (int k = k_lo; k < k_hi; k += 2 * U) {
    load(k + U, bI, bQ);
    reduce(k, aI, aQ);
    if (k + U >= k_hi) break;
    load(k + 2 * U, aI, aQ);
    reduce(k + U, bI, bQ);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < k_hi - k_lo; i += kQuadThreads) {
    float s0 = 0.f, s2 = 0.f;
#pragma unroll
    for (int w = 0; w < nw; ++w) {
      s0 += red[i][w][0];
      s2 += red[i][w][1];
    }
    float* o = Q.part + ((int64_t)(k_lo + i) * gridDim.x + blockIdx.x) * 2;
    o[0] = s0;
    o[1] = s2;
  }
  // publish the partials, then count this CTA in its row
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(Q.cnt + ky, 1) == (int)gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  // the row's last CTA: one warp per height sums the columns' partials
  // (lane-strided, then the fixed shuffle tree: the order does not depend on
  // which CTA came last).  The row's partials are one contiguous block; when
  // it fits, the whole CTA first copies it to shared memory, so the block
  // costs one round trip to L2 instead of one per height.
  const int gx = gridDim.x;
  const int nrow = (k_hi - k_lo) * gx * 2;
  const float* prow = Q.part + (int64_t)k_lo * gx * 2;
  const bool staged = nrow <= kQuadFinal;
  if (staged) {
    for (int i = threadIdx.x; i < nrow; i += kQuadThreads) fin[i] = __ldcg(prow + i);
    __syncthreads();
  }
  for (int i = warp; i < k_hi - k_lo; i += nw) {
    const int k = k_lo + i;
    const float* p = staged ? fin + i * gx * 2 : Q.part + (int64_t)k * gx * 2;
    float a = 0.f, b = 0.f;
    for (int j = lane; j < gx; j += 32) {
      a += staged ? p[2 * j] : __ldcg(p + 2 * j);
      b += staged ? p[2 * j + 1] : __ldcg(p + 2 * j + 1);
    }
    a = warp_sum(a);
    b = warp_sum(b);
    if (lane == 0) {
      float s0 = Q.xi * a, s2 = Q.xiW2 * b;
      if (MODE == KM_LOCAL_LAMBDA) {
        const double* Mi = Q.Minv + 4 * k;
        const float u0 = fmaf((float)Mi[0], s0, (float)Mi[1] * s2);
        const float u2 = fmaf((float)Mi[2], s0, (float)Mi[3] * s2);
        s0 = u0;
        s2 = u2;
      }
      const float2 sg = make_float2(s0, s2);
      reinterpret_cast<float2*>(Q.tab + k)[0] = sg;
      reinterpret_cast<float2*>(Q.tab + (Ns + kTabPad) + (Ns - 1 - k))[0] = sg;
    }
  }
  if (threadIdx.x == 0) Q.cnt[ky] = 0;   // ready for the next launch (stream-ordered)
}

template <typename TV, int MODE>
__global__ void __launch_bounds__(kQuadThreads, 4) k_quad(const TV* __restrict__ x, const double* __restrict__ dinv,
                                                       const float* __restrict__ qw, int64_t nray, int hpc,
                                                       const QuadOut Q, const int* kstop, int step) {
  if (kstop && step >= *kstop) return;
  // x (and the node table the formal solver before may still read) only
  // after the kernel before has finished; the formal solver may start only
  // then too, because in a standalone apply it copies x before its own wait
  pdl_wait();
  pdl_launch_dependents();
  quad_tile<TV, MODE, false>(x, dinv, qw, nray, hpc, Q, blockIdx.y);
}

// k_quad inside GMRES with FP64 vectors, fused with the end of Arnoldi step
// nin.jprev: the first CTA of grid row 0 folds h_{j+1,j}, the Gram row and
// the Givens rotations (Sect. 2.1); rows 1.. form 1/||u|| from the same
// partials in the same order and write x = u / ||u|| as they read u for the
// partials of row blockIdx.y - 1.  Gated by the previous step, since the
// fold itself may end the cycle.
template <int MODE>
__global__ void __launch_bounds__(kQuadThreads) k_quad_norm(double* __restrict__ x, const double* __restrict__ dinv,
                                                            const float* __restrict__ qw, int64_t nray, int hpc,
                                                            const QuadOut Q, const NormIn nin) {
  if (nin.kstop && nin.jprev >= *nin.kstop) return;
  pdl_launch_dependents();
  if (blockIdx.y == 0) {
    if (blockIdx.x == 0)
      arnoldi_fold(nin.part, nin.Gp, nin.ng, nin.hcol, nin.gram, nin.gm, nin.m, nin.jprev, nin.hist, nin.hist_cap);
    return;
  }
  const double inv = arnoldi_inv_norm(nin.part, nin.Gp);
  quad_tile<double, MODE, true>(nullptr, dinv, qw, nray, hpc, Q, blockIdx.y - 1, nin.u, inv, x);
}

// -------------------------------------------------------------- k_staged
struct StagedArgs {
  void* y;                // output (TV), [2][Ns][nray]
  const void* x;          // input (TV): read through the tensor maps; the entry node directly
  const double* dinv;     // Jacobi diagonal (KM_JACOBI)
  const float4* tab;      // [2][Ns + kTabPad] node operands, march-indexed per direction
  const float* r32;       // [nray] phi_hat / |mu|
  const float* t201;      // [Nmu]
  const float* t202;      // [Nmu]
  const float* tile_dt;   // [2][ntile] DELO-linear: sum of dtau / ln 2 over each tile (the tile's slope is 2^-(rsc sum))
  int Ns, Nnu;
  int64_t nray, nd;
  int ngd, ntile, L;      // downward ray groups, tiles per group, steps per tile
  int early;              // 1: x is ready before the quadrature ends (copies may start at once)
  int fail_wait;          // 1: the first wait of CTA 0, warp 0 gives up (failure injection)
  const int* kstop;
  int step;
  int* err;
};

// tensor maps of x and of the Jacobi diagonal, split at the direction
// boundary: [0] the nd downward rays, [1] the upward ones
struct Maps {
  CUtensorMap x[2];
  CUtensorMap d[2];
};

template <typename TV, int FS, int MODE, bool DOWN>
__device__ __forceinline__ void staged_body(const StagedArgs& A, const Maps& M, unsigned char* dsm,
                                            float (*sh)[kMaxT][32], int g, int t, int lane) {
  using C = Cfg<TV, MODE>;
  constexpr int DK = C::DK;
  const int T = A.ntile, Ns = A.Ns, L = A.L;
  const int h = DOWN ? 0 : 1;
  const int64_t hbase = DOWN ? 0 : A.nd;
  const int64_t hext = DOWN ? A.nd : A.nray - A.nd;
  const int c0 = (DOWN ? g : g - A.ngd) * 32;   // first ray of the group within its half
  const bool active = c0 + lane < hext;
  const int64_t r = hbase + (active ? c0 + lane : hext - 1);
  const int j0 = 1 + t * L;                     // first step of the tile (march index)
  const int n1 = max(min(Ns, j0 + L) - j0, 0);
  const int nst = (n1 + DK - 1) / DK;
  unsigned char* wbase = dsm + (size_t)t * kNST * C::STAGE;
  uint64_t* bar = reinterpret_cast<uint64_t*>(dsm + (size_t)T * kNST * C::STAGE) + t * kNST;
  auto issue = [&](int q) {
    const int slot = q % kNST;
    const int c1 = DOWN ? j0 + q * DK : Ns - j0 - (q + 1) * DK;   // lowest height of the box
    unsigned char* s = wbase + slot * C::STAGE;
    mbar_expect_tx(&bar[slot], C::STAGE);
    tma_load_3d(s, &M.x[h], c0, c1, 0, &bar[slot]);
    if (C::JAC) tma_load_3d(s + C::XBYTES, &M.d[h], c0, c1, 0, &bar[slot]);
  };
  if (lane == 0 && nst > 0) {
    for (int s = 0; s < kNST; ++s) mbar_init(&bar[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (A.early)   // x is not written by the kernels before this one
      for (int q = 0; q < kNST && q < nst; ++q) issue(q);
  }
  const int m = (int)(r / A.Nnu);
  const float rsc = __ldg(A.r32 + r);
  const float irsc = 1.0f / rsc;
  const float t201 = __ldg(A.t201 + m), t202 = __ldg(A.t202 + m);
  // the node operands (sigma, written by the quadrature) are read after this
  pdl_wait();
  __syncwarp();
  if (lane == 0 && nst > 0 && !A.early)
    for (int q = 0; q < kNST && q < nst; ++q) issue(q);   // they land while the tile maps are composed
  __syncwarp();
  const float4* tab = A.tab + (size_t)h * (Ns + kTabPad);
  // The recurrence runs on the multipolar components: with S_I = sigma00 +
  // T201 sigma20 and S_Q = T202 sigma20 (Eq. 7-8) and Lambda linear, the
  // formal solution of the ray is I_I = U0 + T201 U2, I_Q = T202 U2, where U0
  // and U2 solve the same recurrence with sigma00 and sigma20 as the source.
  float U0 = 0.f, U2 = 0.f;   // at the tile's inflow node (zero inflow at the entry node)
  if (T > 1) {
    // phase A: the tile's map U_out = E U_in + B (zero inflow gives B)
    if (t < T - 1 && n1 > 0) {
      float4 ring[kRS];
      const float4* pn = tab + j0;
#pragma unroll
      for (int u = 0; u < kRS; ++u) ring[u] = __ldg(pn + u);
      const float4 pp = __ldg(tab + j0 - 1);
      float s0p = pp.x, s2p = pp.y;
      float E = 1.f, B0 = 0.f, B2 = 0.f;
      auto stepA = [&](const float4& op) {
        float e, al, be;
        step_coeffs<FS>(op, rsc, irsc, e, al, be);
        B0 = fmaf(e, B0, fmaf(al, s0p, be * op.x));
        B2 = fmaf(e, B2, fmaf(al, s2p, be * op.y));
        if (FS != RT_FS_DELO_LINEAR) E *= e;
        s0p = op.x;
        s2p = op.y;
      };
      int n = 0;
      for (; n + kRS <= n1; n += kRS) {
#pragma unroll
        for (int u = 0; u < kRS; ++u) {
          const float4 op = ring[u];
          ring[u] = __ldg(pn + kRS + u);   // the table is padded past the last node
          stepA(op);
        }
        pn += kRS;
      }
#pragma unroll
      for (int u = 0; u < kRS; ++u)
        if (n + u < n1) stepA(ring[u]);
      // DELO-linear: the product of the tile's e is exp(-Delta summed over the tile)
      if (FS == RT_FS_DELO_LINEAR) E = ex2_approx(-rsc * __ldg(A.tile_dt + h * T + t));
      sh[0][t][lane] = E;
      sh[1][t][lane] = B0;
      sh[2][t][lane] = B2;
    }
    __syncthreads();
    if (t == 0) {   // phase B: chain the maps into every tile's inflow
      float in0 = 0.f, in1 = 0.f;
      for (int u = 0; u < T; ++u) {
        const bool has = u < T - 1 && 1 + u * L < Ns;
        const float E = has ? sh[0][u][lane] : 1.f;
        const float B0 = has ? sh[1][u][lane] : 0.f, B1 = has ? sh[2][u][lane] : 0.f;
        sh[1][u][lane] = in0;
        sh[2][u][lane] = in1;
        if (has) {
          in0 = fmaf(E, in0, B0);
          in1 = fmaf(E, in1, B1);
        }
      }
    }
    __syncthreads();
    U0 = sh[1][t][lane];
    U2 = sh[2][t][lane];
  }
  const int64_t plane = (int64_t)Ns * A.nray;
  // entry node (tile 0): zero inflow, so y = x there
  if (t == 0 && active) {
    const int64_t o = (int64_t)(DOWN ? 0 : Ns - 1) * A.nray + r;
    const TV* x = reinterpret_cast<const TV*>(A.x);
    TV* y = reinterpret_cast<TV*>(A.y);
    for (int s = 0; s < 2; ++s) {
      if (C::JAC) y[s * plane + o] = (TV)((float)x[s * plane + o] * (float)A.dinv[s * plane + o]);
      else y[s * plane + o] = x[s * plane + o];
    }
  }
  if (nst == 0) return;
  // phase C: re-sweep from the tile's inflow, x from the staged ring
  TV* yI = reinterpret_cast<TV*>(A.y) + (int64_t)(DOWN ? j0 : Ns - 1 - j0) * A.nray + r;
  const int64_t dy = DOWN ? A.nray : -A.nray;
  float4 ring[kRS];
  const float4* pn = tab + j0;
#pragma unroll
  for (int u = 0; u < kRS; ++u) ring[u] = __ldg(pn + u);
  float s0p, s2p;
  {
    const float4 pp = __ldg(tab + j0 - 1);
    s0p = pp.x;
    s2p = pp.y;
  }
  int qfail = -1;
  for (int q = 0; q < nst; ++q) {
    const int slot = q % kNST;
    bool ok;
    if (A.fail_wait && q == 0 && t == 0 && blockIdx.x == 0) ok = false;   // injected: the wait gives up
    else ok = mbar_wait(&bar[slot], (uint32_t)((q / kNST) & 1));
    if (!__all_sync(0xffffffffu, ok)) {
      qfail = q;
      break;
    }
    const TV* xs = reinterpret_cast<const TV*>(wbase + slot * C::STAGE);
    const double* ds = reinterpret_cast<const double*>(wbase + slot * C::STAGE + C::XBYTES);
    const int nb = q * DK;
    auto step = [&](int u) {
      const int ru = u % kRS;
      const int row = DOWN ? u : DK - 1 - u;   // the box runs up in height
      const float4 op = ring[ru];
      ring[ru] = __ldg(pn + kRS + ru);
      if (ru == kRS - 1) pn += kRS;
      float e, al, be;
      step_coeffs<FS>(op, rsc, irsc, e, al, be);
      const float xI = (float)xs[row * 32 + lane], xQ = (float)xs[(DK + row) * 32 + lane];
      float yvI, yvQ;
      if (MODE == KM_LOCAL_LAMBDA) {
        // y = x - (I - beta S): the step without its beta S_k term
        const float t0 = fmaf(e, U0, al * s0p), t2 = fmaf(e, U2, al * s2p);
        yvI = xI - fmaf(t201, t2, t0);
        yvQ = fmaf(-t202, t2, xQ);
        U0 = fmaf(be, op.x, t0);
        U2 = fmaf(be, op.y, t2);
      } else {
        U0 = fmaf(e, U0, fmaf(al, s0p, be * op.x));
        U2 = fmaf(e, U2, fmaf(al, s2p, be * op.y));
        if (MODE == KM_JACOBI) {
          yvI = fmaf(xI, (float)ds[row * 32 + lane], -fmaf(t201, U2, U0));
          yvQ = fmaf(xQ, (float)ds[(DK + row) * 32 + lane], -(t202 * U2));
        } else {
          yvI = xI - fmaf(t201, U2, U0);
          yvQ = fmaf(-t202, U2, xQ);
        }
      }
      s0p = op.x;
      s2p = op.y;
      if (active) {   // evict-first stores: in a large apply, y would push out of L2 the lines of x
                      // that the quadrature left there and other warps have still to read
        __stcs(yI, (TV)yvI);
        __stcs(yI + plane, (TV)yvQ);
      }
      yI += dy;
    };
    if (nb + DK <= n1) {
#pragma unroll
      for (int u = 0; u < DK; ++u) step(u);
    } else {
#pragma unroll
      for (int u = 0; u < DK; ++u)
        if (nb + u < n1) step(u);
    }
    __syncwarp();
    if (lane == 0 && q + kNST < nst) {
      // the warp's reads of this slot come before the copy that overwrites it
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(q + kNST);
    }
    __syncwarp();
  }
  if (qfail >= 0) {
    // a copy did not arrive (or the wait was told to give up): flag it and
    // wait (bounded) for the copies still in flight before the CTA's shared
    // memory is released
    if (lane == 0) atomicExch(A.err, 1);
    const int last = min(nst, qfail + kNST);
    for (int q = qfail; q < last; ++q) mbar_wait(&bar[q % kNST], (uint32_t)((q / kNST) & 1));
  }
}

template <typename TV, int FS, int MODE>
__global__ void __launch_bounds__(32 * kMaxT, RT_STAGED_MINB)
    k_staged(const StagedArgs A, const __grid_constant__ Maps M) {
  extern __shared__ unsigned char dsm_raw[];
  unsigned char* dsm = dsm_raw + ((128 - (smem_u32(dsm_raw) & 127)) & 127);   // 128-byte aligned stages
  __shared__ float sh[3][kMaxT][32];   // per tile: E and B, then the tile's inflow
  __shared__ int gate;
  const int lane = threadIdx.x & 31, t = threadIdx.x >> 5;
  const int g = blockIdx.x;
  if (threadIdx.x == 0) {
    prefetch_tensormap(&M.x[g < A.ngd ? 0 : 1]);
    if (MODE == KM_JACOBI) prefetch_tensormap(&M.d[g < A.ngd ? 0 : 1]);
  }
  if (A.kstop) {   // inside a captured cycle: the step counter is written by the kernels before
    pdl_wait();
    if (threadIdx.x == 0) gate = A.step >= *A.kstop;
    __syncthreads();
    if (gate) return;
  }
  if (g < A.ngd) staged_body<TV, FS, MODE, true>(A, M, dsm, sh, g, t, lane);
  else staged_body<TV, FS, MODE, false>(A, M, dsm, sh, g, t, lane);
}

// ---------------------------------------------------------------- host
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  std::call_once(g_encode_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  });
  return g_encode;
}

template <typename TV, int MODE>
cudaError_t set_smem_attr() {
  const int b = (int)smem_bytes(Cfg<TV, MODE>::WARP, kMaxT);
  cudaError_t e = cudaFuncSetAttribute(k_staged<TV, RT_FS_DELO_LINEAR, MODE>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_staged<TV, RT_FS_IMPLICIT_EULER, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             b);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_staged<TV, RT_FS_TRAPEZOIDAL, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  return e;
}

// 3D tensor map over one direction half of a [2][Ns][nray] vector
bool encode_half(CUtensorMap* tm, const void* base, int64_t first_ray, int64_t nrays, const Problem* P, bool f64,
                 int dk) {
  const cuuint64_t es = f64 ? 8 : 4;
  const cuuint64_t dims[3] = {(cuuint64_t)nrays, (cuuint64_t)P->Ns, 2};
  const cuuint64_t strides[2] = {(cuuint64_t)P->nray * es, (cuuint64_t)P->nray * P->Ns * es};
  const cuuint32_t box[3] = {32, (cuuint32_t)dk, 2};
  const cuuint32_t estr[3] = {1, 1, 1};
  void* addr = const_cast<char*>(static_cast<const char*>(base)) + first_ray * es;
  return encoder()(tm, f64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, addr, dims,
                   strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// the formal solver as a programmatic dependent of the quadrature
template <typename TV, int FS, int MODE>
cudaError_t launch_staged_fs(const Problem* P, const StagedArgs& A, const Maps& M, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(P->ngroups);
  cfg.blockDim = dim3(32 * P->ntile_st);
  cfg.dynamicSmemBytes = smem_bytes(Cfg<TV, MODE>::WARP, P->ntile_st);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_staged<TV, FS, MODE>, A, M);
}

template <typename TV, int MODE>
cudaError_t launch_staged(const Problem* P, const StagedArgs& A, const Maps& M, cudaStream_t st) {
  RT_COUNT(1);
  switch (P->fs) {
    case RT_FS_DELO_LINEAR:
      return launch_staged_fs<TV, RT_FS_DELO_LINEAR, MODE>(P, A, M, st);
    case RT_FS_IMPLICIT_EULER:
      return launch_staged_fs<TV, RT_FS_IMPLICIT_EULER, MODE>(P, A, M, st);
    default:
      return launch_staged_fs<TV, RT_FS_TRAPEZOIDAL, MODE>(P, A, M, st);
  }
}

// The last few tensor-map sets a problem encoded, keyed by the vector
// addresses: encoding costs a few microseconds of host time per apply, which
// a standalone apply would otherwise spend before its first kernel starts.
// A map holds the address and the dimensions only, so an entry stays valid
// for any buffer at that address.
struct MapCache {
  static constexpr int kEntries = 8;
  struct Entry {
    const void* x = nullptr;
    const void* d = nullptr;
    int dk = 0;
    bool f64 = false;
    Maps M;
  } e[kEntries];
  int next = 0;
};

template <typename TV, int MODE>
rt_status staged_maps(Problem* P, const TV* x, Maps* out) {
  constexpr bool f64 = sizeof(TV) == 8;
  const int dk = Cfg<TV, MODE>::DK;
  const void* d = MODE == KM_JACOBI ? static_cast<const void*>(P->dinv) : nullptr;
  if (!P->tma_cache) {
    P->tma_cache = new (std::nothrow) MapCache();
    if (!P->tma_cache) {
      set_error("host allocation failed");
      return RT_ENOMEM;
    }
  }
  MapCache* C = static_cast<MapCache*>(P->tma_cache);
  for (const auto& en : C->e)
    if (en.x == x && en.d == d && en.dk == dk && en.f64 == f64) {
      *out = en.M;
      return RT_OK;
    }
  Maps M;
  memset(&M, 0, sizeof M);
  if (!encode_half(&M.x[0], x, 0, P->nd, P, f64, dk) || !encode_half(&M.x[1], x, P->nd, P->nray - P->nd, P, f64, dk)) {
    set_error("cuTensorMapEncodeTiled failed for the FP32 apply");
    return RT_ECUDA;
  }
  if (MODE == KM_JACOBI && (!encode_half(&M.d[0], P->dinv, 0, P->nd, P, true, dk) ||
                            !encode_half(&M.d[1], P->dinv, P->nd, P->nray - P->nd, P, true, dk))) {
    set_error("cuTensorMapEncodeTiled failed for the Jacobi diagonal");
    return RT_ECUDA;
  }
  MapCache::Entry& en = C->e[C->next];
  C->next = (C->next + 1) % MapCache::kEntries;
  en.x = x;
  en.d = d;
  en.dk = dk;
  en.f64 = f64;
  en.M = M;
  *out = M;
  return RT_OK;
}

template <typename TV, int MODE>
rt_status staged_apply(Problem* P, const TV* x, TV* y, cudaStream_t st, const int* kstop, int step,
                       const NormIn* nin = nullptr, int fail_wait = 0) {
  RT_NVTX("FP32 apply: k_quad + k_staged");
  Maps M;
  RT_TRY((staged_maps<TV, MODE>(P, x, &M)));
  QuadOut Q;
  Q.part = P->qpart;
  Q.cnt = P->qcnt;
  Q.tab = P->stab;
  Q.Minv = P->Minv;
  Q.xi = (float)P->xi;
  Q.xiW2 = (float)(P->xi * P->W2);
  Q.Ns = P->Ns;
  if (nin) {   // FP64 vectors only (staged_apply32): x is written here as u / ||u||
    k_quad_norm<MODE><<<dim3(P->quad_gx, P->quadn_gy + 1), kQuadThreads, 0, st>>>(
        const_cast<double*>(reinterpret_cast<const double*>(x)), P->dinv, P->qw, P->nray, P->quadn_hpc, Q, *nin);
  } else {
    {   // a programmatic dependent of the kernel before
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(P->quad_gx, P->quad_gy);
      cfg.blockDim = dim3(kQuadThreads);
      cfg.stream = st;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      attr[0].val.programmaticStreamSerializationAllowed = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      RT_TRY_CUDA(cudaLaunchKernelEx(&cfg, k_quad<TV, MODE>, x, (const double*)P->dinv, (const float*)P->qw, P->nray,
                                     P->quad_hpc, Q, kstop, step));
    }
  }
  RT_COUNT(1);
  StagedArgs A;
  A.x = x;
  A.y = y;
  A.dinv = P->dinv;
  A.tab = P->stab;
  A.r32 = P->r32;
  A.t201 = P->t201f;
  A.t202 = P->t202f;
  A.tile_dt = P->tile_dt;
  A.Ns = P->Ns;
  A.Nnu = P->Nnu;
  A.nray = P->nray;
  A.nd = P->nd;
  A.ngd = P->ngroups / 2;
  A.ntile = P->ntile_st;
  A.L = (P->Ns - 1 + P->ntile_st - 1) / P->ntile_st;
  A.early = (!nin && !kstop) ? 1 : 0;
  A.fail_wait = fail_wait;
  A.kstop = kstop;
  A.step = step;
  A.err = P->dev_err;
  RT_TRY_CUDA((launch_staged<TV, MODE>(P, A, M, st)));
  RT_TRY_CUDA(cudaGetLastError());
  return RT_OK;
}

// Depth tiles of the staged kernel: the tile count (up to kMaxT, each tile
// at least two stages long) that puts the most warps on the SMs at once,
// min(resident CTAs, ray groups) x tiles; the recurrence is latency-bound,
// so more resident warps beat a grid that fits one wave (measured on the
// N_s = 2000 sweep atmosphere: 16 tiles in 1.3 waves 133 us, 10 tiles in one
// wave 140 us).
int choose_tiles_staged(const Problem* P) {
  int best = 1;
  long long best_warps = -1;
  for (int T = kMaxT; T >= 1; --T) {
    if (T > 1 && (P->Ns - 1) / T < 2 * RT_STAGED_DK) continue;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_staged<float, RT_FS_DELO_LINEAR, KM_PLAIN>, 32 * T,
                                                      smem_bytes(Cfg<float, KM_PLAIN>::WARP, T)) != cudaSuccess) {
      cudaGetLastError();
      occ = 0;
    }
    if (occ <= 0) continue;
    const long long warps = std::min<long long>((long long)occ * P->num_sms, P->ngroups) * T;
    if (warps > best_warps) {
      best_warps = warps;
      best = T;
    }
  }
  return best;
}

}  // namespace

// Prepares the fast FP32 apply of a single problem: quadrature weights, the
// formal solver's node tables, partial sums and row counters, the tile
// count, the kernels' shared-memory opt-in.  Leaves it off (P->staged = 0)
// when the layout does not allow the vector loads and tensor copies, when
// the problem lives in a batch arena, or when RT_NO_TMA=1 is set in the
// environment.
rt_status staged_setup(Problem* P, cudaStream_t st) {
  P->staged = 0;
  if (P->in_arena || P->form == RT_FORM_SIGMA || P->fs == RT_FS_DELO_PARABOLIC) return RT_OK;
  const char* off = std::getenv("RT_NO_TMA");
  if (off && off[0] && off[0] != '0') return RT_OK;
  if ((P->nray % 4) || (P->nd % 4) || !P->dev_err) return RT_OK;
  if (P->Ns > (1 << 24) || P->nray > (1LL << 30)) return RT_OK;
  if (!encoder()) return RT_OK;
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    attr = set_smem_attr<float, KM_PLAIN>();
    if (attr == cudaSuccess) attr = set_smem_attr<double, KM_PLAIN>();
    if (attr == cudaSuccess) attr = set_smem_attr<double, KM_JACOBI>();
    if (attr == cudaSuccess) attr = set_smem_attr<double, KM_LOCAL_LAMBDA>();
  });
  if (attr != cudaSuccess) {
    cudaGetLastError();
    return RT_OK;
  }
  const int Ns = P->Ns, Nmu = P->Nmu, Nnu = P->Nnu;
  const int64_t nray = P->nray;
  // quadrature weights w0 = w_m w_p, w1 = w0 T201_m, w2 = w0 T202_m (the hat weights of Eq. 11-14)
  std::vector<float> qw(3 * nray);
  for (int m = 0; m < Nmu; ++m)
    for (int p = 0; p < Nnu; ++p) {
      const int64_t r = (int64_t)m * Nnu + p;
      const double w0 = 0.5 * P->w_mu[m] * P->w_nu[p];
      qw[r] = (float)w0;
      qw[nray + r] = (float)(w0 * P->t201[m]);
      qw[2 * nray + r] = (float)(w0 * P->t202[m]);
    }
  // node tables, march-indexed: entry j of direction h is node(j) (j downward,
  // Ns-1-j upward) with the interval a step into it crosses; .xy (sigma) are
  // written by the quadrature of every apply
  const int tn = Ns + kTabPad;
  std::vector<float4> tab(2 * (size_t)tn, make_float4(0.f, 0.f, 0.f, 0.f));
  for (int h = 0; h < 2; ++h)
    for (int j = 1; j < Ns; ++j) {
      const int k = h == 0 ? j : Ns - 1 - j;   // node reached by step j
      const double dt = h == 0 ? P->tau[k] - P->tau[k - 1] : P->tau[k + 1] - P->tau[k];
      float4& o = tab[(size_t)h * tn + j];
      if (P->fs == RT_FS_DELO_LINEAR) {
        o.z = (float)(dt / kLn2);
        o.w = (float)(1.0 / dt);
      } else {
        o.z = (float)dt;
      }
    }
  const int64_t nc = nray / 4;
  P->quad_gx = (int)((nc + kQuadThreads - 1) / kQuadThreads);
  const int64_t target = 4LL * P->num_sms;   // CTAs of k_quad: one wave at 4 resident per SM
  const int gy = (int)std::max<int64_t>(1, std::min<int64_t>(Ns, target / P->quad_gx));
  P->quad_hpc = std::min((Ns + gy - 1) / gy, kQuadMaxHeights);
  P->quad_gy = (Ns + P->quad_hpc - 1) / P->quad_hpc;
  // k_quad_norm: taller CTAs, so that the grid is one wave of resident CTAs
  // (each CTA first forms 1/||u|| from the norm partials; a second wave would
  // repeat that serially).  The resident count is the smallest over the
  // three instantiations the solvers launch.  The partial layout depends on
  // quad_gx only.
  P->quadn_hpc = P->quad_hpc;
  int resident = 1 << 30;
  {
    int o[3] = {0, 0, 0};
    bool okq = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o[0], k_quad_norm<KM_PLAIN>, kQuadThreads, 0) ==
                   cudaSuccess &&
               cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o[1], k_quad_norm<KM_JACOBI>, kQuadThreads, 0) ==
                   cudaSuccess &&
               cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o[2], k_quad_norm<KM_LOCAL_LAMBDA>, kQuadThreads, 0) ==
                   cudaSuccess;
    if (!okq) {
      cudaGetLastError();
      resident = 0;
    }
    for (int i = 0; i < 3 && okq; ++i) resident = std::min(resident, o[i]);
  }
  if (resident > 0) {
    const int64_t rows = std::max<int64_t>(1, (int64_t)resident * P->num_sms / P->quad_gx - 1);
    const int h = (int)std::min<int64_t>(kQuadMaxHeights, (Ns + rows - 1) / rows);
    P->quadn_hpc = std::max(P->quad_hpc, h);
  }
  P->quadn_gy = (Ns + P->quadn_hpc - 1) / P->quadn_hpc;
  P->ntile_st = choose_tiles_staged(P);
#ifdef RT_EXPERIMENT
  if (const char* t = std::getenv("RT_STAGED_TILES")) P->ntile_st = std::min(kMaxT, std::max(1, std::atoi(t)));
#endif
  // per depth tile and direction, the sum of the steps' dtau / ln 2 (DELO-linear tile slopes)
  const int T = P->ntile_st, L = (Ns - 1 + T - 1) / T;
  std::vector<float> tdt(2 * (size_t)T, 0.f);
  for (int h = 0; h < 2; ++h)
    for (int t = 0; t < T; ++t) {
      double sum = 0.0;
      for (int j = 1 + t * L; j < std::min(Ns, 1 + (t + 1) * L); ++j) {
        const int k = h == 0 ? j : Ns - 1 - j;
        sum += (h == 0 ? P->tau[k] - P->tau[k - 1] : P->tau[k + 1] - P->tau[k]) / kLn2;
      }
      tdt[(size_t)h * T + t] = (float)sum;
    }
  const int rows = std::max(P->quad_gy, P->quadn_gy);
  RT_TRY_CUDA(dev_alloc(P, (void**)&P->qw, qw.size() * sizeof(float)));
  RT_TRY_CUDA(cudaMemcpyAsync(P->qw, qw.data(), qw.size() * sizeof(float), cudaMemcpyHostToDevice, st));
  RT_TRY_CUDA(dev_alloc(P, (void**)&P->stab, tab.size() * sizeof(float4)));
  RT_TRY_CUDA(cudaMemcpyAsync(P->stab, tab.data(), tab.size() * sizeof(float4), cudaMemcpyHostToDevice, st));
  RT_TRY_CUDA(dev_alloc(P, (void**)&P->qpart, (size_t)Ns * P->quad_gx * 2 * sizeof(float)));
  RT_TRY_CUDA(dev_alloc(P, (void**)&P->tile_dt, tdt.size() * sizeof(float)));
  RT_TRY_CUDA(cudaMemcpyAsync(P->tile_dt, tdt.data(), tdt.size() * sizeof(float), cudaMemcpyHostToDevice, st));
  RT_TRY_CUDA(dev_alloc(P, (void**)&P->qcnt, (size_t)rows * sizeof(int)));
  RT_TRY_CUDA(cudaMemsetAsync(P->qcnt, 0, (size_t)rows * sizeof(int), st));
  RT_TRY_CUDA(cudaStreamSynchronize(st));
  P->staged = 1;
  return RT_OK;
}

bool staged_f64io_ok(const Problem* P, int mode, const void* x, const void* u) {
  if (!P->staged || (reinterpret_cast<uintptr_t>(x) & 15) || (reinterpret_cast<uintptr_t>(u) & 15)) return false;
  if (mode == AM_JACOBI) return !(reinterpret_cast<uintptr_t>(P->dinv) & 15);
  return mode == AM_PLAIN || mode == AM_LOCAL_LAMBDA;
}

// The whole FP32 apply (quadrature with the multipolar components, formal
// solve) through the kernels above, for FP32 vectors or, with f64io, FP64
// vectors (and then, with nin, the input formed as nin->u / ||nin->u||);
// false when they do not apply (nothing launched, *status untouched).
bool staged_apply32(Problem* P, const void* x, void* y, bool f64io, int mode, cudaStream_t st, const int* kstop,
                    int step, rt_status* status, const NormIn* nin) {
  if (!f64io) {
    if (nin || !P->staged || (reinterpret_cast<uintptr_t>(x) & 15) || mode != AM_PLAIN) return false;
    int fail = 0;
    if (!kstop && P->inject_wait_fail > 0) {   // a standalone apply consumes one armed injection
      fail = 1;
      P->inject_wait_fail -= 1;
    }
    *status = staged_apply<float, KM_PLAIN>(P, static_cast<const float*>(x), static_cast<float*>(y), st, kstop,
                                            step, nullptr, fail);
    return true;
  }
  if (!staged_f64io_ok(P, mode, x, nin ? static_cast<const void*>(nin->u) : x)) return false;
  const double* xd = static_cast<const double*>(x);
  double* yd = static_cast<double*>(y);
  switch (mode) {
    case AM_PLAIN:
      *status = staged_apply<double, KM_PLAIN>(P, xd, yd, st, kstop, step, nin);
      return true;
    case AM_JACOBI:
      *status = staged_apply<double, KM_JACOBI>(P, xd, yd, st, kstop, step, nin);
      return true;
    default:
      *status = staged_apply<double, KM_LOCAL_LAMBDA>(P, xd, yd, st, kstop, step, nin);
      return true;
  }
}

void staged_release(Problem* P) {
  delete static_cast<MapCache*>(P->tma_cache);
  P->tma_cache = nullptr;
}

rt_status check_device_flag(Problem* P, cudaStream_t st) {
  if (!P->dev_err) return RT_OK;
  int h = 0;
  RT_TRY_CUDA(cudaMemcpyAsync(&h, P->dev_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  RT_TRY_CUDA(cudaStreamSynchronize(st));
  if (!h) return RT_OK;
  RT_TRY_CUDA(cudaMemsetAsync(P->dev_err, 0, sizeof(int), st));
  RT_TRY_CUDA(cudaStreamSynchronize(st));
  set_error("a device-side wait for a tensor copy gave up; results of the affected applies are invalid");
  return RT_ETIMEOUT;
}

}  // namespace rt

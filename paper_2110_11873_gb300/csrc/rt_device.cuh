// Device code shared by the single-instance kernels (rt_operator.cu) and the
// batched kernels (rt_batch.cu): the quadrature of one height, the formal
// solver's sweep along one ray, the FP32 step coefficients.
#pragma once

#include "rt_common.cuh"

namespace rt {
namespace {

constexpr int kMomThreads = 256;
constexpr int kMaxTiles = 8;     // FP32 kernel: up to 256 threads per CTA (255 registers a lane)
constexpr int kMaxTiles64 = 16;  // FP64 formal solver: depth tiles per ray group (one warp each)
constexpr int kRing = 8;         // prefetch depth of the FP64 formal-solver kernel (steps)
constexpr int kRing32 = 16;      // prefetch depth of the FP32 kernel (one lane carries I and Q)

enum KMode { KM_PLAIN = 0, KM_JACOBI = 1, KM_LOCAL_LAMBDA = 2, KM_RHS = 3 };

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// beta* (coefficient of S_k in I_k) of ray r = m*Nnu + p at height k: the
// beta of the step ending at k; with the DELO-parabolic downwind coefficients
// cg (else NULL) also e_k times the gamma of the step before, whose downwind
// node is k.  col = coef_col(r, ...) and cstride: the table column and row
// length (coef_col).
__device__ __forceinline__ double beta_star(const double* __restrict__ cb, int k, int m, int64_t col,
                                            int64_t cstride, int Ns, int Nh,
                                            const double* __restrict__ ce = nullptr,
                                            const double* __restrict__ cg = nullptr) {
  if (m < Nh) {
    if (k == 0) return 0.0;
    double b = cb[(int64_t)(k - 1) * cstride + col];
    if (cg && k >= 2) b += ce[(int64_t)(k - 1) * cstride + col] * cg[(int64_t)(k - 2) * cstride + col];
    return b;
  }
  if (k == Ns - 1) return 0.0;
  double b = cb[(int64_t)k * cstride + col];
  if (cg && k <= Ns - 3) b += ce[(int64_t)k * cstride + col] * cg[(int64_t)(k + 1) * cstride + col];
  return b;
}

// ----------------------------------------------------------------- K1: T∘J
// One block per height; warp w sums the direction rows m = w, w+8, ...:
// a_m = sum_p w_p z_I(k,m,p), b_m = sum_p w_p z_Q(k,m,p) (one multiply-add
// per element), then J00 += w_m a_m and J20 += w_m (T201_m a_m + T202_m b_m).
// Every lane issues the loads of a whole row before it adds.  MODE:
// KM_PLAIN z = x; KM_JACOBI z = x * dinv; KM_LOCAL_LAMBDA z = x and
// sigma_k <- M_k^{-1} sigma_k.  TI: input vector type, TC: arithmetic type.
constexpr int kRowChunk = 8;   // loads per lane in flight per Stokes parameter

// moments of height k by the whole block (all threads must call it).
// NORM: the input is x * inv, written to xout in the input's precision as
// each element is read (the GMRES normalisation of the batched solver)
template <typename TI, typename TC, int MODE, bool NORM = false>
__device__ __forceinline__ void moments_height(
    const TI* __restrict__ x, const double* __restrict__ dinv, const TC* __restrict__ wnu,
    const TC* __restrict__ wmu, const TC* __restrict__ t201, const TC* __restrict__ t202,
    const double* __restrict__ Minv, int Ns, int Nmu, int Nnu, TC xi, TC xiW2, TC* __restrict__ S, int k,
    double inv = 1.0, TI* __restrict__ xout = nullptr) {
  const int64_t nray = (int64_t)Nmu * Nnu;
  const int64_t oI = (int64_t)k * nray, oQ = ((int64_t)Ns + k) * nray;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int nw = kMomThreads / 32;
  TC j00 = 0, j20 = 0;
  for (int m = warp; m < Nmu; m += nw) {
    const int64_t row = (int64_t)m * Nnu;
    TC aI = 0, aQ = 0;
    for (int p0 = 0; p0 < Nnu; p0 += 32 * kRowChunk) {
      TC vI[kRowChunk], vQ[kRowChunk], wv[kRowChunk];
#pragma unroll
      for (int c = 0; c < kRowChunk; ++c) {
        const int p = p0 + c * 32 + lane;
        const bool ok = p < Nnu;
        const int64_t q = row + (ok ? p : 0);
        if (NORM) {
          TI a = 0, b = 0;
          if (ok) {
            a = (TI)(x[oI + q] * inv);
            b = (TI)(x[oQ + q] * inv);
            xout[oI + q] = a;
            xout[oQ + q] = b;
          }
          vI[c] = (TC)a;
          vQ[c] = (TC)b;
        } else {
          vI[c] = ok ? (TC)x[oI + q] : (TC)0;
          vQ[c] = ok ? (TC)x[oQ + q] : (TC)0;
        }
        wv[c] = ok ? wnu[p] : (TC)0;
        if (MODE == KM_JACOBI && ok) {
          vI[c] *= (TC)dinv[oI + q];
          vQ[c] *= (TC)dinv[oQ + q];
        }
      }
#pragma unroll
      for (int c = 0; c < kRowChunk; ++c) {
        aI = fma(wv[c], vI[c], aI);
        aQ = fma(wv[c], vQ[c], aQ);
      }
    }
    aI = warp_sum(aI);
    aQ = warp_sum(aQ);
    const TC wm = wmu[m];
    j00 = fma(wm, aI, j00);
    j20 = fma(wm, fma(t201[m], aI, t202[m] * aQ), j20);
  }
  __shared__ TC red[2][nw];
  __shared__ TC sig[2];
  if (lane == 0) { red[0][warp] = j00; red[1][warp] = j20; }
  __syncthreads();
  if (threadIdx.x == 0) {
    TC a = 0, b = 0;
    for (int w = 0; w < nw; ++w) { a += red[0][w]; b += red[1][w]; }
    TC s0 = xi * a, s2 = xiW2 * b;
    if (MODE == KM_LOCAL_LAMBDA) {
      const double* Mi = Minv + 4 * k;
      const TC u0 = (TC)Mi[0] * s0 + (TC)Mi[1] * s2;
      const TC u2 = (TC)Mi[2] * s0 + (TC)Mi[3] * s2;
      s0 = u0;
      s2 = u2;
    }
    sig[0] = s0;
    sig[1] = s2;
  }
  __syncthreads();
  for (int m = threadIdx.x; m < Nmu; m += blockDim.x) {
    S[(int64_t)k * Nmu + m] = sig[0] + t201[m] * sig[1];
    S[((int64_t)Ns + k) * Nmu + m] = t202[m] * sig[1];
  }
}

// FP64 quadrature of height k as flat dot products over its rays (the CTA's
// threads stride over r): with the per-ray weights w0 = hat-w_m hat-w_p,
// w1 = w0 T201_m, w2 = w0 T202_m (wray, [3][nray]),
//     J00 = sum_r w0 I_r,   J20 = sum_r (w1 I_r + w2 Q_r),
// then S as in moments_height.  Every FP64 operation is useful work: no
// lane idles on a short row and there is one reduction per height (the FP64
// pipe bounds this kernel).  Any block size that is a multiple of 32.
// WJ (Jacobi mode): wray holds per-element weights [3][Ns][nray], the
// per-ray weights times the inverse diagonal of the element (I, I, Q), so
// the scaling of x costs no operation here.  NORM: the input is x * inv,
// also written to xout (the GMRES normalisation of NormIn).
template <int MODE, bool WJ = false, bool NORM = false>
__device__ __forceinline__ void moments_flat64(const double* __restrict__ x, const double* __restrict__ dinv,
                                               const double* __restrict__ wray, const double* __restrict__ t201,
                                               const double* __restrict__ t202, const double* __restrict__ Minv,
                                               int Ns, int Nmu, int64_t nray, double xi, double xiW2,
                                               double* __restrict__ S, int k, double inv = 1.0,
                                               double* __restrict__ xout = nullptr) {
  const double* __restrict__ xI = x + (int64_t)k * nray;
  const double* __restrict__ xQ = x + ((int64_t)Ns + k) * nray;
  const double* __restrict__ dI = MODE == KM_JACOBI && !WJ ? dinv + (int64_t)k * nray : nullptr;
  const double* __restrict__ dQ = MODE == KM_JACOBI && !WJ ? dinv + ((int64_t)Ns + k) * nray : nullptr;
  const int64_t plane = (int64_t)Ns * nray;
  const double* __restrict__ w0 = WJ ? wray + (int64_t)k * nray : wray;
  const double* __restrict__ w1 = WJ ? w0 + plane : wray + nray;
  const double* __restrict__ w2 = WJ ? w0 + 2 * plane : wray + 2 * nray;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
#pragma unroll 4
  for (int64_t r = threadIdx.x; r < nray; r += blockDim.x) {
    double vI = xI[r], vQ = xQ[r];
    if (NORM) {
      vI *= inv;
      vQ *= inv;
      xout[(int64_t)k * nray + r] = vI;
      xout[((int64_t)Ns + k) * nray + r] = vQ;
    }
    if (MODE == KM_JACOBI && !WJ) {
      vI *= dI[r];
      vQ *= dQ[r];
    }
    a0 = fma(w0[r], vI, a0);
    a1 = fma(w1[r], vI, a1);
    a2 = fma(w2[r], vQ, a2);
  }
  a1 += a2;
  // transposed warp sum: lanes 0-15 get the sum of a0, lanes 16-31 of a1
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool h16 = lane & 16;
  double t = (h16 ? a1 : a0) + __shfl_xor_sync(0xffffffffu, h16 ? a0 : a1, 16);
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  __shared__ double red[2][32];
  __shared__ double sig[2];
  if ((lane & 15) == 0) red[lane >> 4][warp] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = blockDim.x >> 5;
    double j00 = 0.0, j20 = 0.0;
    for (int w = 0; w < nw; ++w) {
      j00 += red[0][w];
      j20 += red[1][w];
    }
    double s0 = xi * j00, s2 = xiW2 * j20;
    if (MODE == KM_LOCAL_LAMBDA) {
      const double* Mi = Minv + 4 * k;
      const double u0 = Mi[0] * s0 + Mi[1] * s2;
      const double u2 = Mi[2] * s0 + Mi[3] * s2;
      s0 = u0;
      s2 = u2;
    }
    sig[0] = s0;
    sig[1] = s2;
  }
  __syncthreads();
  for (int m = threadIdx.x; m < Nmu; m += blockDim.x) {
    S[(int64_t)k * Nmu + m] = sig[0] + t201[m] * sig[1];
    S[((int64_t)Ns + k) * Nmu + m] = t202[m] * sig[1];
  }
}

// --------------------------------------------------------------- K2: Lambda
// FP32 step coefficients from Delta (DELO-linear: Taylor branch below 0.5)
template <int FS>
__device__ __forceinline__ void coeffs32(float D, float& e, float& al, float& be) {
  if (FS == RT_FS_DELO_LINEAR) {
    e = __expf(-D);
    if (D < 0.5f) {
      // beta = D/2 - D^2/6 + D^3/24 - ..., alpha = D/2 - D^2/3 + D^3/8 - ...  (9 terms)
      float b = -1.0f / 3628800.0f, a = -9.0f / 3628800.0f;
      b = fmaf(b, D, 1.0f / 362880.0f);  a = fmaf(a, D, 8.0f / 362880.0f);
      b = fmaf(b, D, -1.0f / 40320.0f);  a = fmaf(a, D, -7.0f / 40320.0f);
      b = fmaf(b, D, 1.0f / 5040.0f);    a = fmaf(a, D, 6.0f / 5040.0f);
      b = fmaf(b, D, -1.0f / 720.0f);    a = fmaf(a, D, -5.0f / 720.0f);
      b = fmaf(b, D, 1.0f / 120.0f);     a = fmaf(a, D, 4.0f / 120.0f);
      b = fmaf(b, D, -1.0f / 24.0f);     a = fmaf(a, D, -3.0f / 24.0f);
      b = fmaf(b, D, 1.0f / 6.0f);       a = fmaf(a, D, 2.0f / 6.0f);
      b = fmaf(b, D, -0.5f);             a = fmaf(a, D, -0.5f);
      be = -b * D;
      al = -a * D;
    } else {
      const float q = __fdividef(1.0f - e, D);
      be = 1.0f - q;
      al = q - e;
    }
  } else if (FS == RT_FS_IMPLICIT_EULER) {
    e = __frcp_rn(1.0f + D);
    al = 0.0f;
    be = D * e;
  } else {
    const float h = 0.5f * D, q = __frcp_rn(1.0f + h);
    e = (1.0f - h) * q;
    al = h * q;
    be = al;
  }
}

struct FormalArgs {
  const void* x;          // input vector (TV)
  const double* dinv;     // Jacobi inverse diagonal (KM_JACOBI)
  const double* ce;       // FP64 coefficient tables [(Ns-1)][nray]
  const double* ca;
  const double* cb;
  const double* cg;       // DELO-parabolic: downwind coefficient table (else NULL)
  int64_t cstride;        // columns of the FP64 tables (coef_col)
  int cshare;             // 1: one column per (|mu|, p) shared by both directions
  const float* dtau32;    // FP32: interval optical depths
  const float* r32;       // FP32: per-ray scale phi_hat/|mu|
  const void* S;          // source functions (TC) [2][Ns][Nmu]
  void* y;                // output vector (TV)
  int Ns, Nmu, Nnu;
  int64_t nray, nd;       // rays per Stokes parameter, downward rays
  int ngd;                // ray groups of downward rays
  int ntile;              // depth tiles per group (warps per CTA)
  double inflow_bottom;   // KM_RHS: I entering at the bottom (mu > 0)
  const int* kstop;       // graph early exit (NULL: run)
  int step;
};

// One lane: NS Stokes parameters (s0 .. s0+NS-1) of ray r, depth steps
// [j0, j1) in marching order (node index j; height k = j for downward rays,
// Ns-1-j for upward rays).  PHASE 0 composes the tile map (E, B) with zero
// inflow; PHASE 2 composes only B (E, a product of the e coefficients, comes
// from a table); PHASE 1 sweeps from the inflow I and writes the output.
// FP64 with FS = RT_FS_DELO_PARABOLIC: each step also takes gamma times S at
// the downwind node (read from the ring, which then holds one node past the
// tile; gamma is 0 on the last interval of a ray).
template <typename TC, typename TV, int FS, int MODE, int PHASE, int NS, int RING>
__device__ __forceinline__ void sweep(const FormalArgs& A, int s0, bool down, int64_t r, int m, bool active, int j0,
                                      int j1, TC (&I)[NS], TC& E) {
  constexpr bool PARA = sizeof(TC) == 8 && FS == RT_FS_DELO_PARABOLIC;
  const int Ns = A.Ns;
  const int64_t nray = A.nray;
  const int64_t plane = (int64_t)Ns * nray;
  const TC* __restrict__ Sm = reinterpret_cast<const TC*>(A.S) + (int64_t)s0 * Ns * A.Nmu + m;
  const int64_t sstride = (int64_t)Ns * A.Nmu;
  const TV* __restrict__ x = reinterpret_cast<const TV*>(A.x) + (int64_t)s0 * plane;
  TV* __restrict__ y = reinterpret_cast<TV*>(A.y) + (int64_t)s0 * plane;
  const double* __restrict__ dinv = A.dinv + (int64_t)s0 * plane;
  const float rs = (sizeof(TC) == 4) ? A.r32[r] : 0.0f;
  const int64_t col = coef_col(r, A.Nmu / 2, A.Nnu, A.cshare), cstride = A.cstride;
  auto height = [&](int j) { return down ? j : Ns - 1 - j; };
  auto interval = [&](int j) { return down ? j - 1 : Ns - 1 - j; };
  TC sp[NS];
#pragma unroll
  for (int q = 0; q < NS; ++q) sp[q] = Sm[q * sstride + (int64_t)height(j0 - 1) * A.Nmu];  // upwind source
  // gamma of the step before j0 (its downwind node is the tile's first node)
  TC gp = 0;
  if (PARA && j0 >= 2) gp = (TC)A.cg[(int64_t)interval(j0 - 1) * cstride + col];
  // register ring of the next RING steps
  TC re[RING], ra[RING], rb[RING], rg[RING], rsv[RING][NS], rx[RING][NS], rd[RING][NS];
  if (PARA) {
#pragma unroll
    for (int u = 0; u < RING; ++u)
#pragma unroll
      for (int q = 0; q < NS; ++q) rsv[u][q] = 0;
  }
  auto load = [&](int u, int j) {
    if (j < j1) {
      const int k = height(j), i = interval(j);
      if (sizeof(TC) == 8) {
        const int64_t c = (int64_t)i * cstride + col;
        re[u] = (TC)A.ce[c];
        ra[u] = (TC)A.ca[c];
        rb[u] = (TC)A.cb[c];
        if (PARA) rg[u] = (TC)A.cg[c];
      } else {
        re[u] = (TC)A.dtau32[i];   // Delta = dtau_i * r_ray; coefficients formed at use
      }
#pragma unroll
      for (int q = 0; q < NS; ++q) {
        rsv[u][q] = Sm[q * sstride + (int64_t)k * A.Nmu];
        if (PHASE == 1 && MODE != KM_RHS) {
          const int64_t o = q * plane + (int64_t)k * nray + r;
          rx[u][q] = (TC)x[o];
          if (MODE == KM_JACOBI) rd[u][q] = (TC)dinv[o];
        }
      }
    } else if (PARA && j == j1 && j < Ns) {
      // the downwind node of the tile's last step
#pragma unroll
      for (int q = 0; q < NS; ++q) rsv[u][q] = Sm[q * sstride + (int64_t)height(j) * A.Nmu];
    }
  };
  auto step = [&](int u, int j) {
    TC e, al, be;
    if (sizeof(TC) == 8) {
      e = re[u];
      al = ra[u];
      be = rb[u];
    } else {
      float ef, af, bf;
      coeffs32<FS>((float)re[u] * rs, ef, af, bf);
      e = (TC)ef;
      al = (TC)af;
      be = (TC)bf;
    }
    if (PHASE == 0) E *= e;
    const int64_t o = (int64_t)height(j) * nray + r;
#pragma unroll
    for (int q = 0; q < NS; ++q) {
      const TC sk = rsv[u][q];
      // beta S_k, plus gamma S_next for DELO-parabolic
      const TC cur = PARA ? fma(be, sk, rg[u] * rsv[(u + 1) % RING][q]) : be * sk;
      if (PHASE != 1) {
        I[q] = fma(e, I[q], fma(al, sp[q], cur));
      } else if (MODE == KM_LOCAL_LAMBDA) {
        // y = (x + beta* S) - I.  DELO-linear: x - (e I_prev + alpha S_prev).
        // DELO-parabolic (beta* = beta + e gamma_prev, gamma_prev S_k being
        // part of I_prev): x - (e (I_prev - gamma_prev S_k) + alpha S_prev + gamma S_next)
        if (PARA) {
          const TC t = fma(e, fma(-gp, sk, I[q]), fma(al, sp[q], rg[u] * rsv[(u + 1) % RING][q]));
          if (active) y[q * plane + o] = (TV)(rx[u][q] - t);
          I[q] = fma(fma(e, gp, be), sk, t);
        } else {
          const TC t = fma(e, I[q], al * sp[q]);
          if (active) y[q * plane + o] = (TV)(rx[u][q] - t);
          I[q] = fma(be, sk, t);
        }
      } else {
        I[q] = fma(e, I[q], fma(al, sp[q], cur));
        if (active) {
          if (MODE == KM_RHS) y[q * plane + o] = (TV)I[q];
          else if (MODE == KM_JACOBI) y[q * plane + o] = (TV)(rx[u][q] * rd[u][q] - I[q]);
          else y[q * plane + o] = (TV)(rx[u][q] - I[q]);
        }
      }
      sp[q] = sk;
    }
    if (PARA) gp = rg[u];
  };
#pragma unroll
  for (int u = 0; u < RING; ++u) load(u, j0 + u);
  int jb = j0;
  // full rounds: every step of the round and every refill is in range, so the
  // round is straight-line code the compiler can interleave across steps
  for (; jb + 2 * RING <= j1; jb += RING) {
#pragma unroll
    for (int u = 0; u < RING; ++u) {
      step(u, jb + u);
      load(u, jb + u + RING);
    }
  }
  for (; jb < j1; jb += RING) {
#pragma unroll
    for (int u = 0; u < RING; ++u) {
      if (jb + u < j1) {
        step(u, jb + u);
        load(u, jb + u + RING);
      }
    }
  }
}

}  // namespace
}  // namespace rt

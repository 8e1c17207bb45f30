// The matrix-free transfer operator of Eq. (19), y = x - Lambda(T(J x)), as
// two kernels per application (Algorithm 1, transposed to the I-form):
//
//   k_moments  (quadrature T∘J, Eq. 11-14 and 7-8): one block per height k
//              reduces the Nmu*Nnu rays of I and Q to J00_k, J20_k, forms
//              sigma_k and writes the source functions S_I(k,m), S_Q(k,m).
//              Each warp owns whole direction rows m, so the quadrature is
//              sum_m w_m T2_m (sum_p w_p x_mp): one multiply-add per element.
//   k_formal   (formal solver Lambda, Eq. 9-10): one thread per (m,p) ray,
//              carrying both Stokes parameters down the depth recurrence
//              I_k = e I_prev + alpha S_prev + beta S_k, and writing
//              y_k = z_k - I_k on the fly.  Neighbouring threads are
//              neighbouring frequencies, so every depth step is a coalesced
//              row access.
//
// FP64 variant: step coefficients (e, alpha, beta) precomputed per
// (interval, |mu|, nu) in FP64 (shared by I, Q and by +-mu).  FP32 variant:
// coefficients recomputed from Delta in FP32 with a Taylor branch for small
// Delta, so the apply streams only x and y.
#include <math.h>

#include "rt_common.cuh"

namespace rt {

namespace {

constexpr int kMomThreads = 256;
constexpr int kFormalThreads = 128;

enum KMode { KM_PLAIN = 0, KM_JACOBI = 1, KM_LOCAL_LAMBDA = 2 };

__device__ __forceinline__ int abs_mu_index(int m, int Nh) { return m < Nh ? Nh - 1 - m : m - Nh; }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ------------------------------------------------------------- setup kernels
// Step coefficients of the formal solvers, FP64, per interval i, |mu| index
// mm and frequency p:  Delta = dtau_i * phi_hat_p / |mu|.
__global__ void k_coeffs64(const double* __restrict__ dtau, const double* __restrict__ phat,
                           const double* __restrict__ absmu, int Ns, int Nh, int Nnu, int fs,
                           double* __restrict__ ce, double* __restrict__ ca, double* __restrict__ cb) {
  const int64_t n = (int64_t)(Ns - 1) * Nh * Nnu;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int p = (int)(t % Nnu);
    const int64_t q = t / Nnu;
    const int mm = (int)(q % Nh);
    const int i = (int)(q / Nh);
    const double D = dtau[i] * phat[p] / absmu[mm];
    double e, al, be;
    if (fs == RT_FS_DELO_LINEAR) {
      if (D < 0.5) {
        // beta = sum_{n>=1} (-1)^{n+1} D^n/(n+1)!,  alpha = sum (-1)^{n+1} n D^n/(n+1)!
        // Horner form, 20 terms (0.5^20/21! ~ 2e-26)
        double b = 0.0, a = 0.0;
        double c = 1.0;
        for (int k = 2; k <= 21; ++k) c /= k;   // c = 1/21!
        // walk n = 20..1 with c_n = 1/(n+1)!
        for (int nn = 20; nn >= 1; --nn) {
          const double sgn = (nn & 1) ? 1.0 : -1.0;
          b = b * D + sgn * c;
          a = a * D + sgn * nn * c;
          c *= (nn + 1);
        }
        be = b * D;
        al = a * D;
        e = exp(-D);
      } else {
        e = exp(-D);
        const double r = -expm1(-D) / D;
        be = 1.0 - r;
        al = r - e;
      }
    } else if (fs == RT_FS_IMPLICIT_EULER) {
      e = 1.0 / (1.0 + D);
      al = 0.0;
      be = D * e;
    } else {
      const double h = 0.5 * D, q2 = 1.0 / (1.0 + h);
      e = (1.0 - h) * q2;
      al = h * q2;
      be = al;
    }
    ce[t] = e;
    ca[t] = al;
    cb[t] = be;
  }
}

// beta* (coefficient of S_k in I_k) of ray (m,p) at height k
__device__ __forceinline__ double beta_star(const double* __restrict__ cb, int k, int m, int p, int Ns,
                                            int Nh, int Nnu) {
  const int mm = abs_mu_index(m, Nh);
  if (m < Nh) return k == 0 ? 0.0 : cb[((int64_t)(k - 1) * Nh + mm) * Nnu + p];
  return k == Ns - 1 ? 0.0 : cb[((int64_t)k * Nh + mm) * Nnu + p];
}

// 2x2 local blocks M_k = Id - J_k Lambda*_k T_k of the sigma-form and their
// inverses, one block per height.
__global__ void __launch_bounds__(kMomThreads) k_local_blocks(const double* __restrict__ cb,
                                                             const double* __restrict__ wray,
                                                             const double* __restrict__ t201,
                                                             const double* __restrict__ t202, int Ns,
                                                             int Nmu, int Nnu, double xi, double W2,
                                                             double* __restrict__ Minv) {
  const int k = blockIdx.x;
  const int Nh = Nmu / 2;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double a0 = 0, a1 = 0, a2 = 0;
  for (int m = warp; m < Nmu; m += nw) {
    double s = 0;
    for (int p = lane; p < Nnu; p += 32) s += wray[m * Nnu + p] * beta_star(cb, k, m, p, Ns, Nh, Nnu);
    s = warp_sum(s);
    a0 += s;
    a1 += t201[m] * s;
    a2 += (t201[m] * t201[m] + t202[m] * t202[m]) * s;
  }
  __shared__ double red[3][32];
  if (lane == 0) { red[0][warp] = a0; red[1][warp] = a1; red[2][warp] = a2; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double b0 = 0, b1 = 0, b2 = 0;
    for (int w = 0; w < nw; ++w) { b0 += red[0][w]; b1 += red[1][w]; b2 += red[2][w]; }
    const double m00 = 1.0 - xi * b0, m01 = -xi * b1, m10 = -xi * W2 * b1, m11 = 1.0 - xi * W2 * b2;
    const double det = m00 * m11 - m01 * m10;
    Minv[4 * k + 0] = m11 / det;
    Minv[4 * k + 1] = -m01 / det;
    Minv[4 * k + 2] = -m10 / det;
    Minv[4 * k + 3] = m00 / det;
  }
}

// inverse Jacobi diagonal (or the diagonal itself) of Id - Lambda T J
__global__ void k_jacobi(const double* __restrict__ cb, const double* __restrict__ wray,
                         const double* __restrict__ t201, const double* __restrict__ t202, int Ns, int Nmu,
                         int Nnu, double xi, double W2, int inverse, double* __restrict__ d) {
  const int Nh = Nmu / 2;
  const int64_t nray = (int64_t)Nmu * Nnu, N = 2 * (int64_t)Ns * nray;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t % nray;
    const int64_t sk = t / nray;
    const int k = (int)(sk % Ns), s = (int)(sk / Ns);
    const int m = (int)(r / Nnu), p = (int)(r % Nnu);
    const double bw = beta_star(cb, k, m, p, Ns, Nh, Nnu) * wray[r];
    const double v = s == 0 ? 1.0 - xi * bw * (1.0 + W2 * t201[m] * t201[m])
                            : 1.0 - xi * W2 * bw * t202[m] * t202[m];
    d[t] = inverse ? 1.0 / v : v;
  }
}

// source functions of the right-hand side: S_I = eps B_k, S_Q = 0
__global__ void k_rhs_source(const double* __restrict__ B, int Ns, int Nmu, double eps, double* __restrict__ S) {
  const int64_t n = (int64_t)Ns * Nmu;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    S[t] = eps * B[t / Nmu];
    S[n + t] = 0.0;
  }
}

// ----------------------------------------------------------------- K1: T∘J
// MODE: KM_PLAIN z = x; KM_JACOBI z = x * dinv; KM_LOCAL_LAMBDA z = x and the
// per-height sigma is replaced by M_k^{-1} sigma.  TI: input vector type,
// TC: compute type of the quadrature.
template <typename TI, typename TC, int MODE>
__global__ void __launch_bounds__(kMomThreads) k_moments(const TI* __restrict__ x, const double* __restrict__ dinv,
                                                         const TC* __restrict__ wray, const TC* __restrict__ t201,
                                                         const TC* __restrict__ t202,
                                                         const double* __restrict__ Minv, int Ns, int Nmu,
                                                         int Nnu, TC xi, TC xiW2, TC* __restrict__ S,
                                                         const int* kstop, int step) {
  if (kstop && step >= *kstop) return;
  const int k = blockIdx.x;
  const int64_t nray = (int64_t)Nmu * Nnu;
  const TI* xI = x + (int64_t)k * nray;
  const TI* xQ = x + ((int64_t)Ns + k) * nray;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  TC j00 = 0, j20 = 0;
  for (int m = warp; m < Nmu; m += nw) {
    TC aI = 0, aQ = 0;
    for (int p = lane; p < Nnu; p += 32) {
      const int idx = m * Nnu + p;
      const TC w = wray[idx];
      TC vI = (TC)xI[idx], vQ = (TC)xQ[idx];
      if (MODE == KM_JACOBI) {
        vI *= (TC)dinv[(int64_t)k * nray + idx];
        vQ *= (TC)dinv[((int64_t)Ns + k) * nray + idx];
      }
      aI += w * vI;
      aQ += w * vQ;
    }
    aI = warp_sum(aI);
    aQ = warp_sum(aQ);
    j00 += aI;
    j20 += t201[m] * aI + t202[m] * aQ;
  }
  __shared__ TC red[2][32];
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

// ------------------------------------------------------------ K2: Lambda, FP64
// MODE: KM_PLAIN y = x - Lambda S;  KM_JACOBI y = x*dinv - Lambda S;
// KM_LOCAL_LAMBDA y = u - Lambda S with u = x + beta* S, which reduces to
// y_k = x_k - (e I_prev + alpha S_prev).
// RHS (rhs != 0): y = Lambda S + t, the boundary inflow included.
template <int MODE>
__global__ void __launch_bounds__(kFormalThreads) k_formal64(
    const double* __restrict__ x, const double* __restrict__ dinv, const double* __restrict__ ce,
    const double* __restrict__ ca, const double* __restrict__ cb, const double* __restrict__ S,
    double* __restrict__ y, int Ns, int Nmu, int Nnu, int rhs, double inflow_bottom, const int* kstop, int step) {
  if (kstop && step >= *kstop) return;
  const int64_t nray = (int64_t)Nmu * Nnu;
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= nray) return;
  const int Nh = Nmu >> 1;
  const int m = (int)(r / Nnu), p = (int)(r - (int64_t)m * Nnu);
  const bool down = m < Nh;
  const int mm = abs_mu_index(m, Nh);
  const int64_t cstr = (int64_t)Nh * Nnu, coff = (int64_t)mm * Nnu + p;
  const int64_t qoff = (int64_t)Ns * nray;
  const double* SI = S + m;
  const double* SQ = S + (int64_t)Ns * Nmu + m;
  const int k0 = down ? 0 : Ns - 1;
  const int dk = down ? 1 : -1;
  double II = (rhs && !down) ? inflow_bottom : 0.0, IQ = 0.0;
  double sIp = SI[(int64_t)k0 * Nmu], sQp = SQ[(int64_t)k0 * Nmu];
  {
    const int64_t o = (int64_t)k0 * nray + r;
    if (rhs) {
      y[o] = II;
      y[qoff + o] = IQ;
    } else if (MODE == KM_JACOBI) {
      y[o] = x[o] * dinv[o];
      y[qoff + o] = x[qoff + o] * dinv[qoff + o];
    } else {
      y[o] = x[o];
      y[qoff + o] = x[qoff + o];
    }
  }
#pragma unroll 4
  for (int j = 1; j < Ns; ++j) {
    const int k = k0 + j * dk;
    const int i = down ? k - 1 : k;
    const int64_t c = (int64_t)i * cstr + coff;
    const double e = ce[c], al = ca[c], be = cb[c];
    const double sI = SI[(int64_t)k * Nmu], sQ = SQ[(int64_t)k * Nmu];
    const int64_t o = (int64_t)k * nray + r;
    if (rhs) {
      II = fma(e, II, fma(al, sIp, be * sI));
      IQ = fma(e, IQ, fma(al, sQp, be * sQ));
      y[o] = II;
      y[qoff + o] = IQ;
    } else if (MODE == KM_LOCAL_LAMBDA) {
      const double tI = fma(e, II, al * sIp), tQ = fma(e, IQ, al * sQp);
      y[o] = x[o] - tI;
      y[qoff + o] = x[qoff + o] - tQ;
      II = fma(be, sI, tI);
      IQ = fma(be, sQ, tQ);
    } else {
      II = fma(e, II, fma(al, sIp, be * sI));
      IQ = fma(e, IQ, fma(al, sQp, be * sQ));
      double zI = x[o], zQ = x[qoff + o];
      if (MODE == KM_JACOBI) {
        zI *= dinv[o];
        zQ *= dinv[qoff + o];
      }
      y[o] = zI - II;
      y[qoff + o] = zQ - IQ;
    }
    sIp = sI;
    sQp = sQ;
  }
}

// ------------------------------------------------------------ K2: Lambda, FP32
// coefficients from Delta in FP32 (DELO-linear: Taylor branch below 0.5)
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
      const float r = (1.0f - e) / D;
      be = 1.0f - r;
      al = r - e;
    }
  } else if (FS == RT_FS_IMPLICIT_EULER) {
    e = 1.0f / (1.0f + D);
    al = 0.0f;
    be = D * e;
  } else {
    const float h = 0.5f * D, q = 1.0f / (1.0f + h);
    e = (1.0f - h) * q;
    al = h * q;
    be = al;
  }
}

template <typename TV, int FS, int MODE>
__global__ void __launch_bounds__(kFormalThreads) k_formal32(
    const TV* __restrict__ x, const double* __restrict__ dinv, const float* __restrict__ dtau,
    const float* __restrict__ rr, const float* __restrict__ S, TV* __restrict__ y, int Ns, int Nmu, int Nnu,
    const int* kstop, int step) {
  if (kstop && step >= *kstop) return;
  const int64_t nray = (int64_t)Nmu * Nnu;
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= nray) return;
  const int Nh = Nmu >> 1;
  const int m = (int)(r / Nnu), p = (int)(r - (int64_t)m * Nnu);
  const bool down = m < Nh;
  const float rp = rr[abs_mu_index(m, Nh) * Nnu + p];
  const int64_t qoff = (int64_t)Ns * nray;
  const float* SI = S + m;
  const float* SQ = S + (int64_t)Ns * Nmu + m;
  const int k0 = down ? 0 : Ns - 1;
  const int dk = down ? 1 : -1;
  float II = 0.f, IQ = 0.f;
  float sIp = SI[(int64_t)k0 * Nmu], sQp = SQ[(int64_t)k0 * Nmu];
  {
    const int64_t o = (int64_t)k0 * nray + r;
    if (MODE == KM_JACOBI) {
      y[o] = (TV)((float)x[o] * (float)dinv[o]);
      y[qoff + o] = (TV)((float)x[qoff + o] * (float)dinv[qoff + o]);
    } else {
      y[o] = x[o];
      y[qoff + o] = x[qoff + o];
    }
  }
#pragma unroll 4
  for (int j = 1; j < Ns; ++j) {
    const int k = k0 + j * dk;
    const int i = down ? k - 1 : k;
    float e, al, be;
    coeffs32<FS>(dtau[i] * rp, e, al, be);
    const float sI = SI[(int64_t)k * Nmu], sQ = SQ[(int64_t)k * Nmu];
    const int64_t o = (int64_t)k * nray + r;
    if (MODE == KM_LOCAL_LAMBDA) {
      const float tI = fmaf(e, II, al * sIp), tQ = fmaf(e, IQ, al * sQp);
      y[o] = (TV)((float)x[o] - tI);
      y[qoff + o] = (TV)((float)x[qoff + o] - tQ);
      II = fmaf(be, sI, tI);
      IQ = fmaf(be, sQ, tQ);
    } else {
      II = fmaf(e, II, fmaf(al, sIp, be * sI));
      IQ = fmaf(e, IQ, fmaf(al, sQp, be * sQ));
      float zI = (float)x[o], zQ = (float)x[qoff + o];
      if (MODE == KM_JACOBI) {
        zI *= (float)dinv[o];
        zQ *= (float)dinv[qoff + o];
      }
      y[o] = (TV)(zI - II);
      y[qoff + o] = (TV)(zQ - IQ);
    }
    sIp = sI;
    sQp = sQ;
  }
}

inline int grid_for(int64_t n, int threads, int cap) {
  int64_t g = (n + threads - 1) / threads;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

// --------------------------------------------------------------- host side
void free_device(Problem* P) {
  void* ptrs[] = {P->ce, P->ca, P->cb, P->wray, P->t201d, P->t202d, P->Bd, P->Minv, P->S, P->S2,
                  P->dtau32, P->r32, P->wray32, P->t201f, P->t202f, P->S32, P->V, P->work, P->dinv,
                  P->work32, P->partials, P->gm, P->bc, P->hist};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  P->ce = P->ca = P->cb = P->wray = P->t201d = P->t202d = P->Bd = P->Minv = P->S = P->S2 = nullptr;
  P->dtau32 = P->r32 = P->wray32 = P->t201f = P->t202f = P->S32 = nullptr;
  P->V = P->work = P->dinv = P->partials = P->hist = nullptr;
  P->work32 = nullptr;
  P->gm = nullptr;
  P->bc = nullptr;
}

template <typename T>
static rt_status upload(T** dst, const std::vector<T>& src, cudaStream_t st) {
  RT_TRY_CUDA(cudaMalloc((void**)dst, src.size() * sizeof(T)));
  RT_TRY_CUDA(cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, st));
  return RT_OK;
}

rt_status setup_device_tables(Problem* P, cudaStream_t st) {
  const int Ns = P->Ns, Nmu = P->Nmu, Nnu = P->Nnu, Nh = P->Nh;
  std::vector<double> dtau(Ns - 1), absmu(Nh), wray((size_t)Nmu * Nnu);
  for (int i = 0; i + 1 < Ns; ++i) dtau[i] = P->tau[i + 1] - P->tau[i];
  for (int mm = 0; mm < Nh; ++mm) absmu[mm] = P->mu[Nh + mm];
  for (int m = 0; m < Nmu; ++m)
    for (int p = 0; p < Nnu; ++p) wray[(size_t)m * Nnu + p] = 0.5 * P->w_mu[m] * P->w_nu[p];
  double *d_dtau = nullptr, *d_phat = nullptr, *d_absmu = nullptr;
  RT_TRY(upload(&d_dtau, dtau, st));
  RT_TRY(upload(&d_phat, P->phi_hat, st));
  RT_TRY(upload(&d_absmu, absmu, st));
  RT_TRY(upload(&P->wray, wray, st));
  RT_TRY(upload(&P->t201d, P->t201, st));
  RT_TRY(upload(&P->t202d, P->t202, st));
  RT_TRY(upload(&P->Bd, P->B, st));
  const size_t nc = (size_t)(Ns - 1) * Nh * Nnu;
  RT_TRY_CUDA(cudaMalloc((void**)&P->ce, nc * sizeof(double)));
  RT_TRY_CUDA(cudaMalloc((void**)&P->ca, nc * sizeof(double)));
  RT_TRY_CUDA(cudaMalloc((void**)&P->cb, nc * sizeof(double)));
  RT_TRY_CUDA(cudaMalloc((void**)&P->Minv, (size_t)Ns * 4 * sizeof(double)));
  RT_TRY_CUDA(cudaMalloc((void**)&P->S, (size_t)2 * Ns * Nmu * sizeof(double)));
  RT_TRY_CUDA(cudaMalloc((void**)&P->S2, (size_t)2 * Ns * Nmu * sizeof(double)));
  k_coeffs64<<<grid_for((int64_t)nc, 256, 8 * P->num_sms), 256, 0, st>>>(d_dtau, d_phat, d_absmu, Ns, Nh, Nnu,
                                                                         P->fs, P->ce, P->ca, P->cb); RT_COUNT(1);
  RT_TRY_CUDA(cudaGetLastError());
  k_local_blocks<<<Ns, kMomThreads, 0, st>>>(P->cb, P->wray, P->t201d, P->t202d, Ns, Nmu, Nnu, P->xi, P->W2,
                                             P->Minv); RT_COUNT(1);
  RT_TRY_CUDA(cudaGetLastError());
  // FP32 tables
  std::vector<float> dtau32(Ns - 1), r32((size_t)Nh * Nnu), wray32(wray.size()), t201f(Nmu), t202f(Nmu);
  for (int i = 0; i + 1 < Ns; ++i) dtau32[i] = (float)dtau[i];
  for (int mm = 0; mm < Nh; ++mm)
    for (int p = 0; p < Nnu; ++p) r32[(size_t)mm * Nnu + p] = (float)(P->phi_hat[p] / absmu[mm]);
  for (size_t t = 0; t < wray.size(); ++t) wray32[t] = (float)wray[t];
  for (int m = 0; m < Nmu; ++m) { t201f[m] = (float)P->t201[m]; t202f[m] = (float)P->t202[m]; }
  RT_TRY(upload(&P->dtau32, dtau32, st));
  RT_TRY(upload(&P->r32, r32, st));
  RT_TRY(upload(&P->wray32, wray32, st));
  RT_TRY(upload(&P->t201f, t201f, st));
  RT_TRY(upload(&P->t202f, t202f, st));
  RT_TRY_CUDA(cudaMalloc((void**)&P->S32, (size_t)2 * Ns * Nmu * sizeof(float)));
  RT_TRY_CUDA(cudaStreamSynchronize(st));
  cudaFree(d_dtau);
  cudaFree(d_phat);
  cudaFree(d_absmu);
  return RT_OK;
}

static int formal_grid(const Problem* P) { return (int)((P->nray + kFormalThreads - 1) / kFormalThreads); }

rt_status op_apply64(Problem* P, const double* x, double* y, int mode, cudaStream_t st, const int* kstop,
                     int step) {
  const double xiW2 = P->xi * P->W2;
  const int g = formal_grid(P);
  const int Ns = P->Ns, Nmu = P->Nmu, Nnu = P->Nnu;
  switch (mode) {
    case AM_PLAIN:
      k_moments<double, double, KM_PLAIN><<<Ns, kMomThreads, 0, st>>>(
          x, nullptr, P->wray, P->t201d, P->t202d, nullptr, Ns, Nmu, Nnu, P->xi, xiW2, P->S, kstop, step); RT_COUNT(1);
      k_formal64<KM_PLAIN><<<g, kFormalThreads, 0, st>>>(x, nullptr, P->ce, P->ca, P->cb, P->S, y, Ns, Nmu, Nnu, 0,
                                                         0.0, kstop, step); RT_COUNT(1);
      break;
    case AM_JACOBI:
      k_moments<double, double, KM_JACOBI><<<Ns, kMomThreads, 0, st>>>(
          x, P->dinv, P->wray, P->t201d, P->t202d, nullptr, Ns, Nmu, Nnu, P->xi, xiW2, P->S, kstop, step); RT_COUNT(1);
      k_formal64<KM_JACOBI><<<g, kFormalThreads, 0, st>>>(x, P->dinv, P->ce, P->ca, P->cb, P->S, y, Ns, Nmu, Nnu, 0,
                                                          0.0, kstop, step); RT_COUNT(1);
      break;
    case AM_LOCAL_LAMBDA:
      k_moments<double, double, KM_LOCAL_LAMBDA><<<Ns, kMomThreads, 0, st>>>(
          x, nullptr, P->wray, P->t201d, P->t202d, P->Minv, Ns, Nmu, Nnu, P->xi, xiW2, P->S, kstop, step); RT_COUNT(1);
      k_formal64<KM_LOCAL_LAMBDA><<<g, kFormalThreads, 0, st>>>(x, nullptr, P->ce, P->ca, P->cb, P->S, y, Ns, Nmu,
                                                                Nnu, 0, 0.0, kstop, step); RT_COUNT(1);
      break;
    default:
      set_error("bad apply mode");
      return RT_EINVAL;
  }
  RT_TRY_CUDA(cudaGetLastError());
  return RT_OK;
}

template <typename TV, int MODE>
static void launch_formal32(Problem* P, const TV* x, TV* y, cudaStream_t st, const int* kstop, int step) {
  const int g = formal_grid(P);
  switch (P->fs) {
    case RT_FS_DELO_LINEAR:
      k_formal32<TV, RT_FS_DELO_LINEAR, MODE><<<g, kFormalThreads, 0, st>>>(
          x, P->dinv, P->dtau32, P->r32, P->S32, y, P->Ns, P->Nmu, P->Nnu, kstop, step); RT_COUNT(1);
      break;
    case RT_FS_IMPLICIT_EULER:
      k_formal32<TV, RT_FS_IMPLICIT_EULER, MODE><<<g, kFormalThreads, 0, st>>>(
          x, P->dinv, P->dtau32, P->r32, P->S32, y, P->Ns, P->Nmu, P->Nnu, kstop, step); RT_COUNT(1);
      break;
    default:
      k_formal32<TV, RT_FS_TRAPEZOIDAL, MODE><<<g, kFormalThreads, 0, st>>>(
          x, P->dinv, P->dtau32, P->r32, P->S32, y, P->Ns, P->Nmu, P->Nnu, kstop, step); RT_COUNT(1);
  }
}

template <typename TV>
static rt_status apply32_impl(Problem* P, const TV* x, TV* y, int mode, cudaStream_t st, const int* kstop,
                              int step) {
  const float xi = (float)P->xi, xiW2 = (float)(P->xi * P->W2);
  const int Ns = P->Ns, Nmu = P->Nmu, Nnu = P->Nnu;
  switch (mode) {
    case AM_PLAIN:
      k_moments<TV, float, KM_PLAIN><<<Ns, kMomThreads, 0, st>>>(x, nullptr, P->wray32, P->t201f, P->t202f, nullptr,
                                                                  Ns, Nmu, Nnu, xi, xiW2, P->S32, kstop, step); RT_COUNT(1);
      launch_formal32<TV, KM_PLAIN>(P, x, y, st, kstop, step);
      break;
    case AM_JACOBI:
      k_moments<TV, float, KM_JACOBI><<<Ns, kMomThreads, 0, st>>>(x, P->dinv, P->wray32, P->t201f, P->t202f,
                                                                   nullptr, Ns, Nmu, Nnu, xi, xiW2, P->S32, kstop,
                                                                   step); RT_COUNT(1);
      launch_formal32<TV, KM_JACOBI>(P, x, y, st, kstop, step);
      break;
    case AM_LOCAL_LAMBDA:
      k_moments<TV, float, KM_LOCAL_LAMBDA><<<Ns, kMomThreads, 0, st>>>(x, nullptr, P->wray32, P->t201f, P->t202f,
                                                                         P->Minv, Ns, Nmu, Nnu, xi, xiW2, P->S32,
                                                                         kstop, step); RT_COUNT(1);
      launch_formal32<TV, KM_LOCAL_LAMBDA>(P, x, y, st, kstop, step);
      break;
    default:
      set_error("bad apply mode");
      return RT_EINVAL;
  }
  RT_TRY_CUDA(cudaGetLastError());
  return RT_OK;
}

rt_status op_apply32(Problem* P, const float* x, float* y, int mode, cudaStream_t st) {
  return apply32_impl<float>(P, x, y, mode, st, nullptr, 0);
}

rt_status op_apply32_f64io(Problem* P, const double* x, double* y, int mode, cudaStream_t st, const int* kstop,
                           int step) {
  return apply32_impl<double>(P, x, y, mode, st, kstop, step);
}

rt_status op_jacobi_inv(Problem* P, double* dinv, cudaStream_t st) {
  k_jacobi<<<grid_for(P->N, 256, 8 * P->num_sms), 256, 0, st>>>(P->cb, P->wray, P->t201d, P->t202d, P->Ns, P->Nmu,
                                                                 P->Nnu, P->xi, P->W2, 1, dinv); RT_COUNT(1);
  RT_TRY_CUDA(cudaGetLastError());
  return RT_OK;
}

rt_status op_rhs(Problem* P, double* b, cudaStream_t st) {
  k_rhs_source<<<grid_for((int64_t)P->Ns * P->Nmu, 256, 4 * P->num_sms), 256, 0, st>>>(P->Bd, P->Ns, P->Nmu, P->eps,
                                                                                      P->S2); RT_COUNT(1);
  k_formal64<KM_PLAIN><<<formal_grid(P), kFormalThreads, 0, st>>>(nullptr, nullptr, P->ce, P->ca, P->cb, P->S2, b,
                                                                  P->Ns, P->Nmu, P->Nnu, 1, P->B[P->Ns - 1],
                                                                  nullptr, 0); RT_COUNT(1);
  RT_TRY_CUDA(cudaGetLastError());
  return RT_OK;
}

// z = P^{-1} v = v + beta* T M^{-1} J v
namespace {
__global__ void k_add_local(const double* __restrict__ v, const double* __restrict__ cb,
                            const double* __restrict__ S, int Ns, int Nmu, int Nnu, double* __restrict__ z) {
  const int Nh = Nmu / 2;
  const int64_t nray = (int64_t)Nmu * Nnu, N = 2 * (int64_t)Ns * nray;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t % nray, sk = t / nray;
    const int k = (int)(sk % Ns), s = (int)(sk / Ns);
    const int m = (int)(r / Nnu), p = (int)(r % Nnu);
    z[t] = v[t] + beta_star(cb, k, m, p, Ns, Nh, Nnu) * S[((int64_t)s * Ns + k) * Nmu + m];
  }
}
}  // namespace

rt_status op_precond_ll(Problem* P, const double* v, double* z, cudaStream_t st) {
  const double xiW2 = P->xi * P->W2;
  k_moments<double, double, KM_LOCAL_LAMBDA><<<P->Ns, kMomThreads, 0, st>>>(
      v, nullptr, P->wray, P->t201d, P->t202d, P->Minv, P->Ns, P->Nmu, P->Nnu, P->xi, xiW2, P->S2, nullptr, 0); RT_COUNT(1);
  k_add_local<<<grid_for(P->N, 256, 8 * P->num_sms), 256, 0, st>>>(v, P->cb, P->S2, P->Ns, P->Nmu, P->Nnu, z); RT_COUNT(1);
  RT_TRY_CUDA(cudaGetLastError());
  return RT_OK;
}

}  // namespace rt

using namespace rt;

extern "C" {

static rt_status check_prob(rt_problem* prob) {
  clear_error();
  if (!prob) {
    set_error("prob is NULL");
    return RT_EINVAL;
  }
  return RT_OK;
}

rt_status rt_apply(rt_problem* prob, const double* x_dev, double* y_dev, void* stream) {
  RT_TRY(check_prob(prob));
  if (!x_dev || !y_dev || x_dev == y_dev) {
    set_error("x_dev and y_dev must be distinct non-NULL device buffers");
    return RT_EINVAL;
  }
  return op_apply64(&prob->P, x_dev, y_dev, AM_PLAIN, as_stream(stream));
}

rt_status rt_apply_f32(rt_problem* prob, const float* x_dev, float* y_dev, void* stream) {
  RT_TRY(check_prob(prob));
  if (!x_dev || !y_dev || (const void*)x_dev == (const void*)y_dev) {
    set_error("x_dev and y_dev must be distinct non-NULL device buffers");
    return RT_EINVAL;
  }
  return op_apply32(&prob->P, x_dev, y_dev, AM_PLAIN, as_stream(stream));
}

rt_status rt_rhs(rt_problem* prob, double* b_dev, void* stream) {
  RT_TRY(check_prob(prob));
  if (!b_dev) {
    set_error("b_dev is NULL");
    return RT_EINVAL;
  }
  return op_rhs(&prob->P, b_dev, as_stream(stream));
}

rt_status rt_jacobi_diag(rt_problem* prob, double* d_dev, void* stream) {
  RT_TRY(check_prob(prob));
  if (!d_dev) {
    set_error("d_dev is NULL");
    return RT_EINVAL;
  }
  Problem* P = &prob->P;
  k_jacobi<<<grid_for(P->N, 256, 8 * P->num_sms), 256, 0, as_stream(stream)>>>(
      P->cb, P->wray, P->t201d, P->t202d, P->Ns, P->Nmu, P->Nnu, P->xi, P->W2, 0, d_dev); RT_COUNT(1);
  RT_TRY_CUDA(cudaGetLastError());
  return RT_OK;
}

rt_status rt_precond_local_lambda(rt_problem* prob, const double* v_dev, double* z_dev, void* stream) {
  RT_TRY(check_prob(prob));
  if (!v_dev || !z_dev || v_dev == z_dev) {
    set_error("v_dev and z_dev must be distinct non-NULL device buffers");
    return RT_EINVAL;
  }
  return op_precond_ll(&prob->P, v_dev, z_dev, as_stream(stream));
}

}  // extern "C"

// The matrix-free transfer operator of Eq. (19), y = x - Lambda(T(J x)), as
// two kernels per application (Algorithm 1, transposed to the I-form):
//
//   k_moments  quadrature T∘J (Eq. 11-14, 7-8): one block per height k
//              reduces the Nmu*Nnu rays of I and Q to J00_k and J20_k with
//              precomputed per-ray weights (w, w T201, w T202), forms sigma_k
//              and writes the source functions S_I(k,m), S_Q(k,m).
//   k_fmapdot, FP64 formal solver as an affine scan over depth tiles:
//   k_fsweep   k_fmapdot forms the offset B of every tile's map but the last
//              as a dot product of setup weights with the tile's node source
//              values (one thread per tile and ray); the units of k_fsweep --
//              (ray group, Stokes parameter, depth tile), one warp and one
//              CTA each, so they spread evenly over the SMs -- chain the maps
//              of the tiles before their own (the slopes E are a setup
//              table) and sweep their tile with the output.
//   k_formal   formal solver Lambda (Eq. 9-10) along every ray, writing
//              y_k = z_k - I_k on the fly.  A CTA owns one group of 32 rays of
//              the same direction sign (so the 32 lanes of a warp read one
//              contiguous row of x per depth step) and splits the depth into
//              `ntile` tiles, one warp each.  With more than one tile the
//              depth recurrence I_k = e I_prev + alpha S_prev + beta S_k is
//              solved as an affine scan: every warp first composes the map
//              I_out = E I_in + B of its tile (phase A), one warp chains the
//              maps over the tiles (phase B), and every warp then re-sweeps
//              its tile from the right inflow (phase C).  Each lane keeps a
//              ring of the next kRing steps' loads in registers so that
//              memory latency overlaps the recurrence.
//
// FP64: step coefficients (e, alpha, beta) are precomputed per (interval,
// ray) in FP64 and streamed; FP64 arithmetic on this GPU is ~70x slower than
// FP32, so the FP64 kernels are built to issue as few FP64 operations as the
// recurrence needs (8 per (k,m,p) for both Stokes parameters).  FP32: the
// coefficients are recomputed from Delta in FP32, so the apply streams only
// x and y.
#include <math.h>

#include <algorithm>
#include <cstdlib>

#include "rt_device.cuh"

namespace rt {

namespace {

// ------------------------------------------------------------- setup kernels
// Step coefficients of the formal solvers, FP64, per interval i and ray r:
// Delta = dtau_i * phi_hat_p / |mu_m|.
// DELO-parabolic (cg != NULL): the DELO-linear coefficients corrected by
// q = int_0^Delta e^{-v} v (v - Delta) dv and the downwind optical path Dn
// (interval i+1 for downward rays, i-1 for upward ones; none on the last
// interval of a ray, where the step stays DELO-linear):
//   alpha += q / (D (D + Dn)),  beta -= q / (D Dn),  gamma = q / (Dn (D + Dn)).
__global__ void k_coeffs64(const double* __restrict__ dtau, const double* __restrict__ rscale, int Ns,
                           int64_t cstride, int shared, int Nh, int Nnu, int fs, double* __restrict__ ce,
                           double* __restrict__ ca, double* __restrict__ cb, double* __restrict__ cg) {
  const int64_t n = (int64_t)(Ns - 1) * cstride;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = t % cstride;
    const int i = (int)(t / cstride);
    // the ray this column stands for (shared columns: the upward ray of that |mu| and p)
    const int64_t r = shared ? ((int64_t)Nh + c / Nnu) * Nnu + c % Nnu : c;
    const double D = dtau[i] * rscale[r];
    double e, al, be;
    if (fs == RT_FS_DELO_LINEAR || fs == RT_FS_DELO_PARABOLIC) {
      e = exp(-D);
      if (D < 0.5) {
        // beta = sum_{n>=1} (-1)^{n+1} D^n/(n+1)!,  alpha = sum (-1)^{n+1} n D^n/(n+1)!
        // Horner form over n = 20..1 (0.5^20/21! ~ 2e-26)
        double b = 0.0, a = 0.0, c = 1.0;
        for (int k = 2; k <= 21; ++k) c /= k;  // 1/21!
        for (int nn = 20; nn >= 1; --nn) {
          const double sgn = (nn & 1) ? 1.0 : -1.0;
          b = b * D + sgn * c;
          a = a * D + sgn * nn * c;
          c *= (nn + 1);
        }
        be = b * D;
        al = a * D;
      } else {
        const double q = -expm1(-D) / D;   // w0 / Delta
        be = 1.0 - q;
        al = q - e;
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
    if (fs == RT_FS_DELO_PARABOLIC) {
      const bool down = (int)(r / Nnu) < Nh;
      const int in = down ? i + 1 : i - 1;
      double ga = 0.0;
      if (in >= 0 && in < Ns - 1) {
        const double Dn = dtau[in] * rscale[r];
        double q;
        if (D < 0.5) {
          // q = -D^3 sum_{j>=0} (-D)^j / (j! (j+2) (j+3)) (0.5^25/25! ~ 1e-33)
          double acc = 0.0, tj = 1.0;
          for (int j = 0; j <= 24; ++j) {
            acc += tj / ((j + 2.0) * (j + 3.0));
            tj *= -D / (j + 1.0);
          }
          q = -acc * D * D * D;
        } else {
          q = D * ((2.0 - D) * al - D * e);
        }
        al += q / (D * (D + Dn));
        be -= q / (D * Dn);
        ga = q / (Dn * (D + Dn));
      }
      cg[t] = ga;
    }
    ce[t] = e;
    ca[t] = al;
    cb[t] = be;
  }
}

// 2x2 local blocks M_k = Id - J_k Lambda*_k T_k of the sigma-form, their
// inverses and their diagonals, one block per height.
__global__ void __launch_bounds__(kMomThreads) k_local_blocks(const double* __restrict__ cb,
                                                             const double* __restrict__ ce,
                                                             const double* __restrict__ cg,
                                                             const double* __restrict__ wray,
                                                             const double* __restrict__ t201,
                                                             const double* __restrict__ t202, int Ns, int Nmu,
                                                             int Nnu, int64_t cstride, int shared, double xi,
                                                             double W2, double* __restrict__ Minv,
                                                             double* __restrict__ Mdiag) {
  const int k = blockIdx.x;
  const int Nh = Nmu / 2;
  const int64_t nray = (int64_t)Nmu * Nnu;
  double a0 = 0, a1 = 0, a2 = 0;
  for (int64_t r = threadIdx.x; r < nray; r += blockDim.x) {
    const int m = (int)(r / Nnu);
    const double s = wray[r] * beta_star(cb, k, m, coef_col(r, Nh, Nnu, shared), cstride, Ns, Nh, ce, cg);
    a0 += s;
    a1 += t201[m] * s;
    a2 += (t201[m] * t201[m] + t202[m] * t202[m]) * s;
  }
  __shared__ double red[3][kMomThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  a0 = warp_sum(a0);
  a1 = warp_sum(a1);
  a2 = warp_sum(a2);
  if (lane == 0) { red[0][warp] = a0; red[1][warp] = a1; red[2][warp] = a2; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double b0 = 0, b1 = 0, b2 = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { b0 += red[0][w]; b1 += red[1][w]; b2 += red[2][w]; }
    const double m00 = 1.0 - xi * b0, m01 = -xi * b1, m10 = -xi * W2 * b1, m11 = 1.0 - xi * W2 * b2;
    const double det = m00 * m11 - m01 * m10;
    Minv[4 * k + 0] = m11 / det;
    Minv[4 * k + 1] = -m01 / det;
    Minv[4 * k + 2] = -m10 / det;
    Minv[4 * k + 3] = m00 / det;
    Mdiag[2 * k + 0] = m00;
    Mdiag[2 * k + 1] = m11;
  }
}

// Jacobi diagonal of Id - Lambda T J, or its inverse
__global__ void k_jacobi(const double* __restrict__ cb, const double* __restrict__ ce, const double* __restrict__ cg,
                         const double* __restrict__ wray,
                         const double* __restrict__ t201, const double* __restrict__ t202, int Ns, int Nmu, int Nnu,
                         int64_t cstride, int shared, double xi, double W2, int inverse, double* __restrict__ d) {
  const int Nh = Nmu / 2;
  const int64_t nray = (int64_t)Nmu * Nnu, N = 2 * (int64_t)Ns * nray;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t % nray;
    const int64_t sk = t / nray;
    const int k = (int)(sk % Ns), s = (int)(sk / Ns);
    const int m = (int)(r / Nnu);
    const double bw = beta_star(cb, k, m, coef_col(r, Nh, Nnu, shared), cstride, Ns, Nh, ce, cg) * wray[r];
    const double v = s == 0 ? 1.0 - xi * bw * (1.0 + W2 * t201[m] * t201[m]) : 1.0 - xi * W2 * bw * t202[m] * t202[m];
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

// source functions of the paper's initial guess sigma^0_0 = 1, sigma^2_0 = 0
// (Sect. 4.2): S_I = 1, S_Q = 0
__global__ void k_unit_source(int Ns, int Nmu, double* __restrict__ S) {
  const int64_t n = (int64_t)Ns * Nmu;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    S[t] = 1.0;
    S[n + t] = 0.0;
  }
}

// z = v + beta* S (the Lambda* T M^{-1} J part of P^{-1} v, S = T M^{-1} J v)
__global__ void k_add_local(const double* __restrict__ v, const double* __restrict__ cb, const double* __restrict__ ce,
                            const double* __restrict__ cg, const double* __restrict__ S,
                            int Ns, int Nmu, int Nnu, int64_t cstride, int shared, double* __restrict__ z,
                            const int* kstop, int step) {
  if (kstop && step >= *kstop) return;
  const int Nh = Nmu / 2;
  const int64_t nray = (int64_t)Nmu * Nnu, N = 2 * (int64_t)Ns * nray;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t % nray, sk = t / nray;
    const int k = (int)(sk % Ns), s = (int)(sk / Ns);
    const int m = (int)(r / Nnu);
    z[t] = v[t] + beta_star(cb, k, m, coef_col(r, Nh, Nnu, shared), cstride, Ns, Nh, ce, cg) *
                      S[((int64_t)s * Ns + k) * Nmu + m];
  }
}


template <typename TI, typename TC, int MODE>
__global__ void __launch_bounds__(kMomThreads) k_moments(
    const TI* __restrict__ x, const double* __restrict__ dinv, const TC* __restrict__ wnu,
    const TC* __restrict__ wmu, const TC* __restrict__ t201, const TC* __restrict__ t202,
    const double* __restrict__ Minv, int Ns, int Nmu, int Nnu, TC xi, TC xiW2, TC* __restrict__ S,
    const int* kstop, int step) {
  if (kstop && step >= *kstop) return;
  moments_height<TI, TC, MODE>(x, dinv, wnu, wmu, t201, t202, Minv, Ns, Nmu, Nnu, xi, xiW2, S, blockIdx.x);
}

// FP64 quadrature, one CTA per height (flat over the rays); WJ: Jacobi mode
// with the per-element weights of k_jacobi_weights in place of wray
constexpr int kMom64Threads = 512;
template <int MODE, bool WJ = false>
__global__ void __launch_bounds__(kMom64Threads) k_moments64(
    const double* __restrict__ x, const double* __restrict__ dinv, const double* __restrict__ wray,
    const double* __restrict__ t201, const double* __restrict__ t202, const double* __restrict__ Minv, int Ns,
    int Nmu, int64_t nray, double xi, double xiW2, double* __restrict__ S, const int* kstop, int step) {
  if (kstop && step >= *kstop) return;
  moments_flat64<MODE, WJ>(x, dinv, wray, t201, t202, Minv, Ns, Nmu, nray, xi, xiW2, S, blockIdx.x);
}

// GMRES (NormIn): block 0 ends Arnoldi step nin.jprev (fold and Givens
// rotations, Sect. 2.1); blocks 1..Ns normalise u into x = u / ||u|| while
// forming the quadrature of x (Eq. 11-14) for height blockIdx.x - 1
template <int MODE, bool WJ>
__global__ void __launch_bounds__(kMom64Threads) k_moments64_norm(
    double* __restrict__ x, const double* __restrict__ dinv, const double* __restrict__ wray,
    const double* __restrict__ t201, const double* __restrict__ t202, const double* __restrict__ Minv, int Ns,
    int Nmu, int64_t nray, double xi, double xiW2, double* __restrict__ S, const NormIn nin) {
  if (nin.kstop && nin.jprev >= *nin.kstop) return;
  pdl_wait();   // the last block pass's w and partials
  if (blockIdx.x == 0) {
    arnoldi_fold(nin.part, nin.Gp, nin.ng, nin.hcol, nin.gram, nin.gm, nin.m, nin.jprev, nin.hist, nin.hist_cap);
    return;
  }
  const double inv = arnoldi_inv_norm(nin.part, nin.Gp);
  moments_flat64<MODE, WJ, true>(nin.u, dinv, wray, t201, t202, Minv, Ns, Nmu, nray, xi, xiW2, S, blockIdx.x - 1,
                                 inv, x);
}

// wjac[q][k][r] = wray[q][r] * D^-1 of element (k, r): Stokes I for q = 0, 1
// and Q for q = 2 (the quadrature weights of the Jacobi-mode apply)
__global__ void k_jacobi_weights(const double* __restrict__ wray, const double* __restrict__ dinv, int Ns,
                                 int64_t nray, double* __restrict__ wjac) {
  const int64_t plane = (int64_t)Ns * nray;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < plane; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i % nray;
    wjac[i] = wray[r] * dinv[i];
    wjac[plane + i] = wray[nray + r] * dinv[i];
    wjac[2 * plane + i] = wray[2 * nray + r] * dinv[plane + i];
  }
}

// grid: NSPLIT * ngroups CTAs (ray group g, and with NSPLIT = 2 the Stokes
// parameter s = blockIdx.x % 2 -- with NSPLIT = 1 one lane carries I and Q);
// block: 32 * ntile threads (warp t = depth tile t)
template <typename TC, typename TV, int FS, int MODE, int NSPLIT, int RING, int MAXT>
__global__ void __launch_bounds__(32 * MAXT) k_formal(const FormalArgs A) {
  constexpr int NS = 2 / NSPLIT;   // Stokes parameters per lane
  if (A.kstop && A.step >= *A.kstop) return;
  const int lane = threadIdx.x & 31, t = threadIdx.x >> 5;
  const int s0 = NSPLIT == 2 ? (blockIdx.x & 1) : 0;
  const int g = NSPLIT == 2 ? (blockIdx.x >> 1) : blockIdx.x;
  const bool down = g < A.ngd;
  const int64_t base = down ? (int64_t)g * 32 : A.nd + (int64_t)(g - A.ngd) * 32;
  const int64_t end = down ? A.nd : A.nray;
  const bool active = base + lane < end;
  const int64_t r = active ? base + lane : end - 1;
  const int m = (int)(r / A.Nnu);
  const int Ns = A.Ns;
  const int T = A.ntile;
  const int L = (Ns - 1 + T - 1) / T;   // steps per tile
  const int j0 = 1 + t * L;
  const int j1 = min(Ns, j0 + L);
  __shared__ TC sh[1 + NS][MAXT][32];   // per tile: E and B, then the tile's inflow
  TC I[NS];
#pragma unroll
  for (int q = 0; q < NS; ++q) I[q] = (MODE == KM_RHS && !down && s0 + q == 0) ? (TC)A.inflow_bottom : (TC)0;
  if (T > 1) {
    // phase A: tile maps (the last tile's map is not needed)
    if (t < T - 1 && j0 < j1) {
      TC E = 1, B[NS];
#pragma unroll
      for (int q = 0; q < NS; ++q) B[q] = 0;
      sweep<TC, TV, FS, MODE, 0, NS, RING>(A, s0, down, r, m, active, j0, j1, B, E);
      sh[0][t][lane] = E;
#pragma unroll
      for (int q = 0; q < NS; ++q) sh[1 + q][t][lane] = B[q];
    }
    __syncthreads();
    // phase B: inflow of every tile
    if (t == 0) {
      TC in[NS];
#pragma unroll
      for (int q = 0; q < NS; ++q) in[q] = I[q];
      for (int u = 0; u < T; ++u) {
        const bool has = u < T - 1 && 1 + u * L < Ns;
        const TC E = has ? sh[0][u][lane] : (TC)1;
#pragma unroll
        for (int q = 0; q < NS; ++q) {
          const TC B = has ? sh[1 + q][u][lane] : (TC)0;
          sh[1 + q][u][lane] = in[q];
          if (has) in[q] = fma(E, in[q], B);
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NS; ++q) I[q] = sh[1 + q][t][lane];
  }
  // entry node (tile 0): the inflow itself
  if (t == 0 && active) {
    const int k0 = down ? 0 : Ns - 1;
    const TV* __restrict__ x = reinterpret_cast<const TV*>(A.x);
    TV* __restrict__ y = reinterpret_cast<TV*>(A.y);
#pragma unroll
    for (int q = 0; q < NS; ++q) {
      const int64_t o = (int64_t)(s0 + q) * Ns * A.nray + (int64_t)k0 * A.nray + r;
      if (MODE == KM_RHS) y[o] = (TV)I[q];
      else if (MODE == KM_JACOBI) y[o] = (TV)((TC)x[o] * (TC)A.dinv[o]);
      else y[o] = x[o];
    }
  }
  // phase C: sweep with the true inflow
  if (j0 < j1) {
    TC E = 1;
    sweep<TC, TV, FS, MODE, 1, NS, RING>(A, s0, down, r, m, active, j0, j1, I, E);
  }
}

// launch_pdl with a multi-dimensional grid and block
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl_shape(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t st,
                                    Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

inline int grid_for(int64_t n, int threads, int cap) {
  int64_t g = (n + threads - 1) / threads;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

// --------------------------------------------------------------- host side
cudaError_t poison_fill(void* p, size_t bytes) {
  const char* e = std::getenv("RT_POISON");
  if (!e || e[0] != '1' || g_capturing || !p || !bytes) return cudaSuccess;
  cudaError_t r = cudaMemset(p, 0xFF, bytes);
  if (r == cudaSuccess) r = cudaDeviceSynchronize();
  return r;
}

cudaError_t dev_alloc(Problem* P, void** p, size_t bytes) {
  cudaError_t e = P->alloc ? P->alloc->alloc(p, bytes) : cudaMalloc(p, bytes);
  return e == cudaSuccess ? poison_fill(*p, bytes) : e;
}

void dev_free(Problem* P, void* p) {
  if (!p) return;
  if (P->alloc) P->alloc->release(p);
  else cudaFree(p);
}

void free_device(Problem* P) {
  void* ptrs[] = {P->ce,     P->ca,    P->cb,     P->wray,   P->wI2,  P->wQ2,   P->t201d, P->t202d,
                  P->Bd,     P->Minv,  P->S,      P->S2,     P->dtau32, P->r32, P->wray32, P->wI2f,
                  P->wQ2f,   P->t201f, P->t202f,  P->S32,    P->V,    P->work,  P->dinv,  P->work32,
                  P->partials, P->gm,  P->bc,     P->hist,  P->dev_err, P->bpart, P->qw, P->stab, P->qpart, P->qcnt, P->tile_dt, P->Mdiag, P->Ibuf, P->cg,
                  P->Etile, P->Bmap, P->Asig, P->Mpre, P->Mtri, P->Mscr, P->wjac, P->Kmap};
  for (void* p : ptrs)
    if (p) dev_free(P, p);
  P->ce = P->ca = P->cb = P->wray = P->wI2 = P->wQ2 = P->t201d = P->t202d = P->Bd = P->Minv = P->S = P->S2 = nullptr;
  P->dtau32 = P->r32 = P->wray32 = P->wI2f = P->wQ2f = P->t201f = P->t202f = P->S32 = nullptr;
  P->V = P->work = P->dinv = P->partials = P->hist = P->bpart = nullptr;
  P->work32 = nullptr;
  P->gm = nullptr;
  P->bc = nullptr;
  P->dev_err = nullptr;
  P->qw = P->qpart = nullptr;
  P->stab = nullptr;
  P->qcnt = nullptr;
  P->tile_dt = nullptr;
  staged_release(P);
  P->Mdiag = P->Ibuf = P->cg = P->Etile = P->Bmap = P->Kmap = nullptr;
  P->Asig = P->Mpre = P->Mtri = P->Mscr = P->wjac = nullptr;
  P->asig_ready = 0;
  P->mpre_kind = 0;
  P->staged = 0;
}

template <typename T>
static rt_status upload(Problem* P, T** dst, const std::vector<T>& src, cudaStream_t st) {
  RT_TRY_CUDA(dev_alloc(P, (void**)dst, src.size() * sizeof(T)));
  RT_TRY_CUDA(cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, st));
  return RT_OK;
}

// Depth tiles per ray group.  FP64: the formal solver's warp units spread
// evenly over the SMs, so an SM carries ceil(units / SMs) of them.  A step
// costs a sweep unit 4 FP64 operations; an SM retires one FP64 warp
// operation in about kFp64OpCycles, while one warp alone needs about
// kFp64StepCycles per step (the dependent chain through I; both measured on
// GB300), and the sweep takes the longer of the two.  The map offsets cost 2
// independent FMAs per tile node and ray (pipe time only).  T minimises the
// sum.  FP32: tiles are cheap, so aim
// at about 16 warps per SM with tiles of at least 2*kRing steps.
constexpr double kFp64OpCycles = 20.0, kFp64StepCycles = 600.0;
static int choose_tiles64(const Problem* P) {
  const int64_t sms = P->num_sms, groups = 2LL * P->ngroups;
  auto kernel = [&](int64_t units, double ops) {
    return std::max((double)((units + sms - 1) / sms) * ops * kFp64OpCycles, kFp64StepCycles);
  };
  int best = 1;
  double best_cost = 1e300;
  for (int T = 1; T <= kMaxTiles64; ++T) {
    const int L = (P->Ns - 1 + T - 1) / T;
    if (T > 1 && L < 2 * kRing) break;
    const double maps = (double)(T - 1) * P->nray * (L + 2) * 2.0 / 32.0 / (double)sms * kFp64OpCycles;
    const double cost = L * kernel(groups * T, 4.0) + maps;
    if (cost < best_cost * 0.97) {
      best_cost = cost;
      best = T;
    }
  }
  return best;
}

// the ray of lane `lane` in ray group g (groups 0..ngd-1 downward); lanes
// past the direction's last ray take that ray and are inactive
__device__ __forceinline__ void group_ray(const FormalArgs& A, int g, int lane, int64_t& r, int& m, bool& down,
                                          bool& active) {
  down = g < A.ngd;
  const int64_t base = down ? (int64_t)g * 32 : A.nd + (int64_t)(g - A.ngd) * 32;
  const int64_t end = down ? A.nd : A.nray;
  active = base + lane < end;
  r = active ? base + lane : end - 1;
  m = (int)(r / A.Nnu);
}

// slope of tile t's map for every ray, E = product of the e coefficients of
// its steps in marching order: Etile[t][r], t < T-1 (setup)
__global__ void k_etile(const double* __restrict__ ce, int Ns, int64_t nray, int64_t nd, int T, int64_t cstride,
                        int shared, int Nh, int Nnu, double* __restrict__ Etile) {
  const int L = (Ns - 1 + T - 1) / T;
  const int64_t n = (int64_t)(T - 1) * nray;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(i / nray);
    const int64_t r = i % nray;
    const bool down = r < nd;
    const int j0 = 1 + t * L, j1 = min(Ns, j0 + L);
    const int64_t col = coef_col(r, Nh, Nnu, shared);
    double E = 1.0;
    for (int j = j0; j < j1; ++j) E *= ce[(int64_t)(down ? j - 1 : Ns - 1 - j) * cstride + col];
    Etile[i] = E;
  }
}

// Weights of the map offsets of the formal solver (Eq. 9-10 marched over a
// depth tile).  With zero inflow the tile recurrence
// I_j = e_j I_{j-1} + alpha_j S_{j-1} + beta_j S_j (+ gamma_j S_{j+1}) ends at
// B = sum_j P_j (alpha_j S_{j-1} + beta_j S_j + gamma_j S_{j+1}), P_j the
// product of the e of the tile's later steps, so B is a fixed linear form in
// the source values at the tile's nodes j0-1 .. j1:
//     B(t, r, s) = sum_n K[t][n][r] S_s(node j0 - 1 + n, m(r)).
// k_kmap builds K at setup (one backward pass per tile and ray); the map
// kernel is then one independent FMA per node instead of a dependent
// recurrence.  K[t][n][r], n < L + 2.
__global__ void k_kmap(const double* __restrict__ ce, const double* __restrict__ ca, const double* __restrict__ cb,
                       const double* __restrict__ cg, int Ns, int64_t nray, int64_t nd, int T, int64_t cstride,
                       int shared, int Nh, int Nnu, double* __restrict__ K) {
  const int L = (Ns - 1 + T - 1) / T;
  const int64_t n = (int64_t)(T - 1) * nray;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(i / nray);
    const int64_t r = i % nray;
    const bool down = r < nd;
    const int j0 = 1 + t * L, j1 = min(Ns, j0 + L);
    double* __restrict__ Kt = K + (int64_t)t * (L + 2) * nray + r;
    for (int q = 0; q < L + 2; ++q) Kt[(int64_t)q * nray] = 0.0;
    const int64_t col = coef_col(r, Nh, Nnu, shared);
    double Pj = 1.0;   // product of e over the steps after j
    for (int j = j1 - 1; j >= j0; --j) {
      const int64_t c = (int64_t)(down ? j - 1 : Ns - 1 - j) * cstride + col;
      const int q = j - j0 + 1;   // local index of node j
      Kt[(int64_t)q * nray] += Pj * cb[c];
      Kt[(int64_t)(q - 1) * nray] += Pj * ca[c];
      if (cg) Kt[(int64_t)(q + 1) * nray] += Pj * cg[c];
      Pj *= ce[c];
    }
  }
}

// the map offsets B of tiles t < T-1 for both Stokes parameters, written as
// Bmap[g * 2 + s][t][lane] for the sweep kernel.  A CTA takes 32 rays of one
// tile (x) and splits the tile's nodes over kMapSlices thread rows (y), so
// many loads are in flight; the rows' partial sums are added in a fixed order.
constexpr int kMapSlices = 8;
__global__ void __launch_bounds__(32 * kMapSlices) k_fmapdot(const FormalArgs A, const double* __restrict__ K,
                                                             double* __restrict__ Bmap) {
  if (A.kstop && A.step >= *A.kstop) return;
  pdl_wait();   // the source values of the quadrature before
  const int Ns = A.Ns, T = A.ntile, L = (Ns - 1 + T - 1) / T;
  const int64_t nray = A.nray;
  const int t = blockIdx.y;
  const int64_t r = (int64_t)blockIdx.x * 32 + threadIdx.x;
  const bool valid = r < nray;
  const int64_t rc = valid ? r : nray - 1;
  const double* __restrict__ S = reinterpret_cast<const double*>(A.S);
  const int64_t sQ = (int64_t)Ns * A.Nmu;
  const bool down = rc < A.nd;
  const int m = (int)(rc / A.Nnu);
  const int j0 = 1 + t * L, jend = min(Ns - 1, j0 + L);   // nodes j0-1 .. jend
  const double* __restrict__ Kt = K + (int64_t)t * (L + 2) * nray + rc;
  double bI = 0.0, bQ = 0.0;
  for (int j = j0 - 1 + (int)threadIdx.y; j <= jend; j += kMapSlices) {
    const double k = Kt[(int64_t)(j - j0 + 1) * nray];
    const int64_t o = (int64_t)(down ? j : Ns - 1 - j) * A.Nmu + m;
    bI = fma(k, S[o], bI);
    bQ = fma(k, S[sQ + o], bQ);
  }
  __shared__ double red[2][kMapSlices][32];
  red[0][threadIdx.y][threadIdx.x] = bI;
  red[1][threadIdx.y][threadIdx.x] = bQ;
  __syncthreads();
  if (threadIdx.y < 2 && valid) {
    double b = 0.0;
#pragma unroll
    for (int y = 0; y < kMapSlices; ++y) b += red[threadIdx.y][y][threadIdx.x];
    const int64_t rr = down ? r : r - A.nd;
    const int g = (int)(rr / 32) + (down ? 0 : A.ngd), lane = (int)(rr % 32);
    Bmap[((size_t)(2 * g + threadIdx.y) * (T - 1) + t) * 32 + lane] = b;
  }
}

// tile t of ray group g, Stokes s: inflow from the boundary through the maps
// of tiles 0..t-1, then the sweep with the output; unit u = (g * 2 + s) * T + t
template <int FS, int MODE>
__global__ void __launch_bounds__(32, FS == RT_FS_DELO_PARABOLIC ? 12 : 16) k_fsweep(const FormalArgs A, const double* __restrict__ Bmap,
                                               const double* __restrict__ Etile) {
  if (A.kstop && A.step >= *A.kstop) return;
  // A programmatic dependent of k_fmapdot.  It never releases its own
  // dependents early: the block passes after it read the basis vector v_j,
  // which this apply's quadrature wrote, before their wait, and that is safe
  // because they start only once every CTA here has exited -- after this
  // wait, hence after the quadrature and the tile maps finished.
  pdl_wait();
  const int T = A.ntile, L = (A.Ns - 1 + T - 1) / T;
  const int u = blockIdx.x, lane = threadIdx.x;
  const int t = u % T, gs = u / T, s0 = gs & 1;
  int64_t r;
  int m;
  bool down, active;
  group_ray(A, gs >> 1, lane, r, m, down, active);
  const int Ns = A.Ns;
  double I[1] = {(MODE == KM_RHS && !down && s0 == 0) ? A.inflow_bottom : 0.0};
  for (int tt = 0; tt < t; ++tt)
    I[0] = fma(Etile[(size_t)tt * A.nray + r], I[0], Bmap[((size_t)gs * (T - 1) + tt) * 32 + lane]);
  if (t == 0 && active) {   // entry node: the inflow itself
    const int64_t o = (int64_t)s0 * Ns * A.nray + (int64_t)(down ? 0 : Ns - 1) * A.nray + r;
    const double* __restrict__ x = reinterpret_cast<const double*>(A.x);
    double* __restrict__ y = reinterpret_cast<double*>(A.y);
    if (MODE == KM_RHS) y[o] = I[0];
    else if (MODE == KM_JACOBI) y[o] = x[o] * A.dinv[o];
    else y[o] = x[o];
  }
  const int j0 = 1 + t * L, j1 = min(Ns, j0 + L);
  if (j0 < j1) {
    double E = 1.0;
    sweep<double, double, FS, MODE, 1, 1, kRing>(A, s0, down, r, m, active, j0, j1, I, E);
  }
}

static int choose_tiles32(const Problem* P) {
  const int64_t want = (8LL * P->num_sms + P->ngroups - 1) / P->ngroups;
  int T = want < 1 ? 1 : (int)(want > kMaxTiles ? kMaxTiles : want);
  while (T > 1 && (P->Ns - 1) / T < 2 * kRing32) --T;
  return T;
}

rt_status setup_device_tables(Problem* P, cudaStream_t st) {
  const int Ns = P->Ns, Nmu = P->Nmu, Nnu = P->Nnu, Nh = P->Nh;
  const int64_t nray = P->nray;
  P->nd = (int64_t)Nh * Nnu;
  const int ngd = (int)((P->nd + 31) / 32);
  P->ngroups = 2 * ngd;
  P->ntile64 = choose_tiles64(P);
#ifdef RT_EXPERIMENT
  if (const char* t = std::getenv("RT_TILES64")) P->ntile64 = std::min(kMaxTiles64, std::max(1, std::atoi(t)));
#endif
  P->ntile32 = choose_tiles32(P);
  std::vector<double> dtau(Ns - 1), rscale(nray), w0(3 * nray), wnu(P->w_nu), wmu(Nmu);
  for (int m = 0; m < Nmu; ++m) wmu[m] = 0.5 * P->w_mu[m];
  for (int i = 0; i + 1 < Ns; ++i) dtau[i] = P->tau[i + 1] - P->tau[i];
  for (int m = 0; m < Nmu; ++m)
    for (int p = 0; p < Nnu; ++p) {
      const size_t r = (size_t)m * Nnu + p;
      rscale[r] = P->phi_hat[p] / fabs(P->mu[m]);
      w0[r] = 0.5 * P->w_mu[m] * P->w_nu[p];
      w0[nray + r] = w0[r] * P->t201[m];       // the J20 weights of I and Q
      w0[2 * nray + r] = w0[r] * P->t202[m];
    }
  double *d_dtau = nullptr, *d_rs = nullptr;
  // the two temporaries are returned on every path (in an arena a leaked
  // block would fragment the memory of later instances)
  struct Temps {
    Problem* P;
    cudaStream_t st;
    double** a;
    double** b;
    ~Temps() {
      if (*a || *b) cudaStreamSynchronize(st);
      dev_free(P, *a);
      dev_free(P, *b);
    }
  } temps{P, st, &d_dtau, &d_rs};
  RT_TRY(upload(P, &d_dtau, dtau, st));
  RT_TRY(upload(P, &d_rs, rscale, st));
  RT_TRY(upload(P, &P->wray, w0, st));
  RT_TRY(upload(P, &P->wI2, wnu, st));   // spectral weights hat-w_p
  RT_TRY(upload(P, &P->wQ2, wmu, st));   // angular weights hat-w_m
  RT_TRY(upload(P, &P->t201d, P->t201, st));
  RT_TRY(upload(P, &P->t202d, P->t202, st));
  RT_TRY(upload(P, &P->Bd, P->B, st));
  // the step coefficients depend on |mu| only unless the scheme has a
  // downwind term: one table column per (|mu|, p) then serves both directions
  P->cshare = P->fs != RT_FS_DELO_PARABOLIC;
  P->cstride = P->cshare ? nray / 2 : nray;
  const size_t nc = (size_t)(Ns - 1) * P->cstride;
  RT_TRY_CUDA(dev_alloc(P, (void**)&P->ce, nc * sizeof(double)));
  RT_TRY_CUDA(dev_alloc(P, (void**)&P->ca, nc * sizeof(double)));
  RT_TRY_CUDA(dev_alloc(P, (void**)&P->cb, nc * sizeof(double)));
  RT_TRY_CUDA(dev_alloc(P, (void**)&P->Minv, (size_t)Ns * 4 * sizeof(double)));
  RT_TRY_CUDA(dev_alloc(P, (void**)&P->S, (size_t)2 * Ns * Nmu * sizeof(double)));
  RT_TRY_CUDA(dev_alloc(P, (void**)&P->S2, (size_t)2 * Ns * Nmu * sizeof(double)));
  if (P->fs == RT_FS_DELO_PARABOLIC) RT_TRY_CUDA(dev_alloc(P, (void**)&P->cg, nc * sizeof(double)));
  k_coeffs64<<<grid_for((int64_t)nc, 256, 8 * P->num_sms), 256, 0, st>>>(d_dtau, d_rs, Ns, P->cstride, P->cshare,
                                                                         Nh, Nnu, P->fs, P->ce, P->ca, P->cb, P->cg);
  RT_COUNT(1);
  RT_TRY_CUDA(cudaGetLastError());
  if (P->ntile64 > 1) {   // the FP64 formal solver's tile slopes and map buffer
    const int T = P->ntile64;
    RT_TRY_CUDA(dev_alloc(P, (void**)&P->Etile, (size_t)(T - 1) * nray * sizeof(double)));
    const size_t nb = (size_t)2 * P->ngroups * (T - 1) * 32;
    RT_TRY_CUDA(dev_alloc(P, (void**)&P->Bmap, nb * sizeof(double)));
    RT_TRY_CUDA(cudaMemsetAsync(P->Bmap, 0, nb * sizeof(double), st));   // lanes past a direction's last ray
    const int L = (Ns - 1 + T - 1) / T;
    const int64_t nk = (int64_t)(T - 1) * (L + 2) * nray;
    RT_TRY_CUDA(dev_alloc(P, (void**)&P->Kmap, (size_t)nk * sizeof(double)));
    k_kmap<<<grid_for((int64_t)(T - 1) * nray, 256, 8 * P->num_sms), 256, 0, st>>>(
        P->ce, P->ca, P->cb, P->cg, Ns, nray, P->nd, T, P->cstride, P->cshare, Nh, Nnu, P->Kmap);
    RT_COUNT(1);
    k_etile<<<grid_for((int64_t)(T - 1) * nray, 256, 8 * P->num_sms), 256, 0, st>>>(
        P->ce, Ns, nray, P->nd, T, P->cstride, P->cshare, Nh, Nnu, P->Etile);
    RT_COUNT(1);
    RT_TRY_CUDA(cudaGetLastError());
  }
  RT_TRY_CUDA(dev_alloc(P, (void**)&P->Mdiag, (size_t)Ns * 2 * sizeof(double)));
  k_local_blocks<<<Ns, kMomThreads, 0, st>>>(P->cb, P->ce, P->cg, P->wray, P->t201d, P->t202d, Ns, Nmu, Nnu,
                                             P->cstride, P->cshare, P->xi, P->W2, P->Minv, P->Mdiag);
  RT_COUNT(1);
  if (P->form == RT_FORM_SIGMA) RT_TRY_CUDA(dev_alloc(P, (void**)&P->Ibuf, (size_t)P->N * sizeof(double)));
  RT_TRY_CUDA(cudaGetLastError());
  // FP32 tables
  std::vector<float> dtau32(Ns - 1), r32(nray), w032(nray), wI32(Nnu), wQ32(Nmu), t201f(Nmu), t202f(Nmu);
  for (int i = 0; i + 1 < Ns; ++i) dtau32[i] = (float)dtau[i];
  for (int64_t r = 0; r < nray; ++r) {
    r32[r] = (float)rscale[r];
    w032[r] = (float)w0[r];
  }
  for (int p = 0; p < Nnu; ++p) wI32[p] = (float)wnu[p];
  for (int m = 0; m < Nmu; ++m) wQ32[m] = (float)wmu[m];
  for (int m = 0; m < Nmu; ++m) { t201f[m] = (float)P->t201[m]; t202f[m] = (float)P->t202[m]; }
  RT_TRY(upload(P, &P->dtau32, dtau32, st));
  RT_TRY(upload(P, &P->r32, r32, st));
  RT_TRY(upload(P, &P->wray32, w032, st));
  RT_TRY(upload(P, &P->wI2f, wI32, st));
  RT_TRY(upload(P, &P->wQ2f, wQ32, st));
  RT_TRY(upload(P, &P->t201f, t201f, st));
  RT_TRY(upload(P, &P->t202f, t202f, st));
  RT_TRY_CUDA(dev_alloc(P, (void**)&P->S32, (size_t)2 * Ns * Nmu * sizeof(float)));
  RT_TRY_CUDA(dev_alloc(P, (void**)&P->dev_err, sizeof(int)));
  RT_TRY_CUDA(cudaMemsetAsync(P->dev_err, 0, sizeof(int), st));
  RT_TRY_CUDA(cudaStreamSynchronize(st));
  return staged_setup(P, st);
}

static FormalArgs formal_args(const Problem* P, const void* x, void* y, const void* S, int ntile, const int* kstop,
                              int step) {
  FormalArgs A;
  A.x = x;
  A.dinv = P->dinv;
  A.ce = P->ce;
  A.ca = P->ca;
  A.cb = P->cb;
  A.cg = P->cg;
  A.cstride = P->cstride;
  A.cshare = P->cshare;
  A.dtau32 = P->dtau32;
  A.r32 = P->r32;
  A.S = S;
  A.y = y;
  A.Ns = P->Ns;
  A.Nmu = P->Nmu;
  A.Nnu = P->Nnu;
  A.nray = P->nray;
  A.nd = P->nd;
  A.ngd = P->ngroups / 2;
  A.ntile = ntile;
  A.inflow_bottom = P->B[P->Ns - 1];
  A.kstop = kstop;
  A.step = step;
  return A;
}

template <int FS, int MODE>
static void formal64_units(const Problem* P, const FormalArgs& A, cudaStream_t st) {
  const int T = P->ntile64, groups = 2 * P->ngroups;
  if (T > 1) {
    launch_pdl_shape(k_fmapdot, dim3((unsigned)((P->nray + 31) / 32), (unsigned)(T - 1)), dim3(32, kMapSlices), st,
                     A, (const double*)P->Kmap, P->Bmap);
    RT_COUNT(1);
  }
  launch_pdl_shape(k_fsweep<FS, MODE>, dim3(groups * T), dim3(32), st, A, (const double*)P->Bmap,
                   (const double*)P->Etile);
  RT_COUNT(1);
}

template <int MODE>
static void launch_formal64(const Problem* P, const double* x, double* y, const double* S, cudaStream_t st,
                            const int* kstop, int step) {
  const FormalArgs A = formal_args(P, x, y, S, P->ntile64, kstop, step);
  if (P->fs == RT_FS_DELO_PARABOLIC) formal64_units<RT_FS_DELO_PARABOLIC, MODE>(P, A, st);
  else formal64_units<0, MODE>(P, A, st);
}

void formal64_lambda(Problem* P, const double* S, double* I_out, double inflow_bottom, cudaStream_t st,
                     const int* kstop, int step) {
  FormalArgs A = formal_args(P, nullptr, I_out, S, P->ntile64, kstop, step);
  A.inflow_bottom = inflow_bottom;
  if (P->fs == RT_FS_DELO_PARABOLIC) formal64_units<RT_FS_DELO_PARABOLIC, KM_RHS>(P, A, st);
  else formal64_units<0, KM_RHS>(P, A, st);
}

template <typename TV, int MODE>
static void launch_formal32(const Problem* P, const TV* x, TV* y, cudaStream_t st, const int* kstop, int step) {
  const FormalArgs A = formal_args(P, x, y, P->S32, P->ntile32, kstop, step);
  const int g = P->ngroups, b = 32 * P->ntile32;
  switch (P->fs) {
    case RT_FS_DELO_LINEAR:
      k_formal<float, TV, RT_FS_DELO_LINEAR, MODE, 1, kRing32, kMaxTiles><<<g, b, 0, st>>>(A); RT_COUNT(1);
      break;
    case RT_FS_IMPLICIT_EULER:
      k_formal<float, TV, RT_FS_IMPLICIT_EULER, MODE, 1, kRing32, kMaxTiles><<<g, b, 0, st>>>(A); RT_COUNT(1);
      break;
    default:
      k_formal<float, TV, RT_FS_TRAPEZOIDAL, MODE, 1, kRing32, kMaxTiles><<<g, b, 0, st>>>(A); RT_COUNT(1);
  }
}

rt_status op_apply64(Problem* P, const double* x, double* y, int mode, cudaStream_t st, const int* kstop, int step,
                     const NormIn* nin) {
  RT_NVTX("operator apply FP64");
  if (P->form == RT_FORM_SIGMA) {
    if (nin) {
      set_error("the fused normalisation needs the I-form");
      return RT_EINVAL;
    }
    return op_apply_sigma(P, x, y, mode, st, kstop, step);
  }
  const double xiW2 = P->xi * P->W2;
  const int Ns = P->Ns, Nmu = P->Nmu;
  if (nin) {   // GMRES: x = u / ||u|| formed by the quadrature kernel
    double* xw = const_cast<double*>(x);
    switch (mode) {
      case AM_PLAIN:
        RT_TRY_CUDA(launch_pdl(k_moments64_norm<KM_PLAIN, false>, Ns + 1, kMom64Threads, st,
            xw, nullptr, P->wray, P->t201d, P->t202d, nullptr, Ns, Nmu, P->nray, P->xi, xiW2, P->S, *nin));
        break;
      case AM_JACOBI:
        if (P->wjac)
          RT_TRY_CUDA(launch_pdl(k_moments64_norm<KM_JACOBI, true>, Ns + 1, kMom64Threads, st,
              xw, nullptr, P->wjac, P->t201d, P->t202d, nullptr, Ns, Nmu, P->nray, P->xi, xiW2, P->S, *nin));
        else
          RT_TRY_CUDA(launch_pdl(k_moments64_norm<KM_JACOBI, false>, Ns + 1, kMom64Threads, st,
              xw, P->dinv, P->wray, P->t201d, P->t202d, nullptr, Ns, Nmu, P->nray, P->xi, xiW2, P->S, *nin));
        break;
      case AM_LOCAL_LAMBDA:
        RT_TRY_CUDA(launch_pdl(k_moments64_norm<KM_LOCAL_LAMBDA, false>, Ns + 1, kMom64Threads, st,
            xw, nullptr, P->wray, P->t201d, P->t202d, P->Minv, Ns, Nmu, P->nray, P->xi, xiW2, P->S, *nin));
        break;
      default:
        set_error("bad apply mode");
        return RT_EINVAL;
    }
    RT_COUNT(1);
    switch (mode) {
      case AM_PLAIN: launch_formal64<KM_PLAIN>(P, x, y, P->S, st, kstop, step); break;
      case AM_JACOBI: launch_formal64<KM_JACOBI>(P, x, y, P->S, st, kstop, step); break;
      default: launch_formal64<KM_LOCAL_LAMBDA>(P, x, y, P->S, st, kstop, step); break;
    }
    RT_TRY_CUDA(cudaGetLastError());
    return RT_OK;
  }
  switch (mode) {
    case AM_PLAIN:
      k_moments64<KM_PLAIN><<<Ns, kMom64Threads, 0, st>>>(x, nullptr, P->wray, P->t201d, P->t202d, nullptr, Ns, Nmu,
                                                          P->nray, P->xi, xiW2, P->S, kstop, step); RT_COUNT(1);
      launch_formal64<KM_PLAIN>(P, x, y, P->S, st, kstop, step);
      break;
    case AM_JACOBI:
      if (P->wjac)
        k_moments64<KM_JACOBI, true><<<Ns, kMom64Threads, 0, st>>>(x, nullptr, P->wjac, P->t201d, P->t202d, nullptr,
                                                                   Ns, Nmu, P->nray, P->xi, xiW2, P->S, kstop, step);
      else
        k_moments64<KM_JACOBI><<<Ns, kMom64Threads, 0, st>>>(x, P->dinv, P->wray, P->t201d, P->t202d, nullptr, Ns,
                                                             Nmu, P->nray, P->xi, xiW2, P->S, kstop, step);
      RT_COUNT(1);
      launch_formal64<KM_JACOBI>(P, x, y, P->S, st, kstop, step);
      break;
    case AM_LOCAL_LAMBDA:
      k_moments64<KM_LOCAL_LAMBDA><<<Ns, kMom64Threads, 0, st>>>(x, nullptr, P->wray, P->t201d, P->t202d, P->Minv,
                                                                 Ns, Nmu, P->nray, P->xi, xiW2, P->S, kstop, step);
      RT_COUNT(1);
      launch_formal64<KM_LOCAL_LAMBDA>(P, x, y, P->S, st, kstop, step);
      break;
    default:
      set_error("bad apply mode");
      return RT_EINVAL;
  }
  RT_TRY_CUDA(cudaGetLastError());
  return RT_OK;
}

template <typename TV>
static rt_status apply32_impl(Problem* P, const TV* x, TV* y, int mode, cudaStream_t st, const int* kstop, int step,
                              const NormIn* nin = nullptr) {
  RT_NVTX("operator apply FP32");
  if (P->fs == RT_FS_DELO_PARABOLIC) {
    set_error("the DELO-parabolic formal solver is FP64 only (use rt_apply, FP64 solvers)");
    return RT_EINVAL;
  }
  if (P->form == RT_FORM_SIGMA) {
    // the sigma-form operator has no FP32 variant: the solvers use the FP64 one
    if (sizeof(TV) == 8)
      return op_apply_sigma(P, reinterpret_cast<const double*>(x), reinterpret_cast<double*>(y), mode, st, kstop,
                            step);
    set_error("the sigma-form operator is FP64 only (use rt_apply)");
    return RT_EINVAL;
  }
  rt_status s = RT_OK;
  if (staged_apply32(P, x, y, sizeof(TV) == 8, mode, st, kstop, step, &s, nin)) return s;
  if (nin) {
    set_error("internal: the fused GMRES normalisation needs the staged FP32 apply");
    return RT_EINVAL;
  }
  const float xi = (float)P->xi, xiW2 = (float)(P->xi * P->W2);
  const int Ns = P->Ns, Nmu = P->Nmu, Nnu = P->Nnu;
  switch (mode) {
    case AM_PLAIN:
      k_moments<TV, float, KM_PLAIN><<<Ns, kMomThreads, 0, st>>>(x, nullptr, P->wI2f, P->wQ2f, P->t201f,
                                                                  P->t202f, nullptr, Ns, Nmu, Nnu, xi, xiW2, P->S32,
                                                                  kstop, step); RT_COUNT(1);
      launch_formal32<TV, KM_PLAIN>(P, x, y, st, kstop, step);
      break;
    case AM_JACOBI:
      k_moments<TV, float, KM_JACOBI><<<Ns, kMomThreads, 0, st>>>(x, P->dinv, P->wI2f, P->wQ2f, P->t201f,
                                                                   P->t202f, nullptr, Ns, Nmu, Nnu, xi, xiW2, P->S32,
                                                                   kstop, step); RT_COUNT(1);
      launch_formal32<TV, KM_JACOBI>(P, x, y, st, kstop, step);
      break;
    case AM_LOCAL_LAMBDA:
      k_moments<TV, float, KM_LOCAL_LAMBDA><<<Ns, kMomThreads, 0, st>>>(x, nullptr, P->wI2f, P->wQ2f,
                                                                         P->t201f, P->t202f, P->Minv, Ns, Nmu, Nnu,
                                                                         xi, xiW2, P->S32, kstop, step); RT_COUNT(1);
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
                           int step, const NormIn* nin) {
  return apply32_impl<double>(P, x, y, mode, st, kstop, step, nin);
}

rt_status op_jacobi_inv(Problem* P, double* dinv, cudaStream_t st) {
  if (P->form == RT_FORM_SIGMA) return op_jacobi_sigma(P, dinv, 1, st);
  k_jacobi<<<grid_for(P->N, 256, 8 * P->num_sms), 256, 0, st>>>(P->cb, P->ce, P->cg, P->wray, P->t201d, P->t202d,
                                                                 P->Ns, P->Nmu, P->Nnu, P->cstride, P->cshare, P->xi,
                                                                 P->W2, 1, dinv);
  RT_COUNT(1);
  RT_TRY_CUDA(cudaGetLastError());
  return RT_OK;
}

rt_status op_jacobi_weights(Problem* P, cudaStream_t st) {
  if (P->form != RT_FORM_I) return RT_OK;
  const int64_t plane = (int64_t)P->Ns * P->nray;
  if (!P->wjac) RT_TRY_CUDA(dev_alloc(P, (void**)&P->wjac, 3 * (size_t)plane * sizeof(double)));
  k_jacobi_weights<<<grid_for(plane, 256, 8 * P->num_sms), 256, 0, st>>>(P->wray, P->dinv, P->Ns, P->nray, P->wjac);
  RT_COUNT(1);
  RT_TRY_CUDA(cudaGetLastError());
  return RT_OK;
}

rt_status op_rhs(Problem* P, double* b, cudaStream_t st) {
  RT_NVTX("right-hand side");
  if (P->form == RT_FORM_SIGMA) return op_rhs_sigma(P, b, st);
  k_rhs_source<<<grid_for((int64_t)P->Ns * P->Nmu, 256, 4 * P->num_sms), 256, 0, st>>>(P->Bd, P->Ns, P->Nmu, P->eps,
                                                                                      P->S2); RT_COUNT(1);
  launch_formal64<KM_RHS>(P, nullptr, b, P->S2, st, nullptr, 0);
  RT_TRY_CUDA(cudaGetLastError());
  return RT_OK;
}

rt_status op_x0_paper(Problem* P, double* x, cudaStream_t st) {
  RT_NVTX("initial guess of the paper");
  if (P->form == RT_FORM_SIGMA) return op_x0_paper_sigma(P, x, st);
  // I = Lambda(T sigma) + t: the formal solve of the right-hand side with
  // S_I = 1 in place of eps B
  k_unit_source<<<grid_for((int64_t)P->Ns * P->Nmu, 256, 4 * P->num_sms), 256, 0, st>>>(P->Ns, P->Nmu, P->S2);
  RT_COUNT(1);
  launch_formal64<KM_RHS>(P, nullptr, x, P->S2, st, nullptr, 0);
  RT_TRY_CUDA(cudaGetLastError());
  return RT_OK;
}

// z = P^{-1} v = v + beta* T M^{-1} J v
rt_status op_precond_ll(Problem* P, const double* v, double* z, cudaStream_t st, const int* kstop, int step) {
  if (P->form == RT_FORM_SIGMA) return op_precond_sigma(P, v, z, st, kstop, step);
  const double xiW2 = P->xi * P->W2;
  k_moments64<KM_LOCAL_LAMBDA><<<P->Ns, kMom64Threads, 0, st>>>(v, nullptr, P->wray, P->t201d, P->t202d, P->Minv,
                                                                P->Ns, P->Nmu, P->nray, P->xi, xiW2, P->S2, kstop,
                                                                step); RT_COUNT(1);
  k_add_local<<<grid_for(P->N, 256, 8 * P->num_sms), 256, 0, st>>>(v, P->cb, P->ce, P->cg, P->S2, P->Ns, P->Nmu,
                                                                    P->Nnu, P->cstride, P->cshare, z, kstop, step);
  RT_COUNT(1);
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
  RT_NVTX("rt_jacobi_diag");
  RT_TRY(check_prob(prob));
  if (!d_dev) {
    set_error("d_dev is NULL");
    return RT_EINVAL;
  }
  Problem* P = &prob->P;
  if (P->form == RT_FORM_SIGMA) return op_jacobi_sigma(P, d_dev, 0, as_stream(stream));
  k_jacobi<<<grid_for(P->N, 256, 8 * P->num_sms), 256, 0, as_stream(stream)>>>(
      P->cb, P->ce, P->cg, P->wray, P->t201d, P->t202d, P->Ns, P->Nmu, P->Nnu, P->cstride, P->cshare, P->xi, P->W2, 0,
      d_dev);
  RT_COUNT(1);
  RT_TRY_CUDA(cudaGetLastError());
  return RT_OK;
}

rt_status rt_precond_local_lambda(rt_problem* prob, const double* v_dev, double* z_dev, void* stream) {
  RT_NVTX("rt_precond_local_lambda");
  RT_TRY(check_prob(prob));
  if (!v_dev || !z_dev || v_dev == z_dev) {
    set_error("v_dev and z_dev must be distinct non-NULL device buffers");
    return RT_EINVAL;
  }
  return op_precond_ll(&prob->P, v_dev, z_dev, as_stream(stream));
}

rt_status rt_precond_stationary(rt_problem* prob, int32_t kind, double omega, const double* v_dev, double* z_dev,
                                void* stream) {
  RT_NVTX("rt_precond_stationary");
  RT_TRY(check_prob(prob));
  if (!v_dev || !z_dev || v_dev == z_dev) {
    set_error("v_dev and z_dev must be distinct non-NULL device buffers");
    return RT_EINVAL;
  }
  if (kind != RT_PREC_SOR && kind != RT_PREC_SSOR) {
    set_error("kind must be RT_PREC_SOR or RT_PREC_SSOR");
    return RT_EINVAL;
  }
  RT_TRY(op_dense_precond_build(&prob->P, kind, omega, as_stream(stream)));
  return op_dense_precond_apply(&prob->P, v_dev, z_dev, as_stream(stream));
}

}  // extern "C"

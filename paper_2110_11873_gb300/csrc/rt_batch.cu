// Batched uneven instances and the serving loop.
//
// Many atmospheres of different sizes are solved together by restarted
// GMRES(m) in lock-step: every phase of an Arnoldi step (quadrature, formal
// solve, each MGS pass, Givens update) is ONE persistent launch over all
// resident instances; the normalisation of a new basis vector happens in
// the next step's quadrature launch.  Each launch walks a device-resident
// work list -- (instance, height) items for the quadrature, (instance, ray
// group, Stokes) items for the formal solver, (instance, vector chunk) items
// for the vector kernels, instances for the scalar updates -- so the grid is
// fixed, the whole restart cycle is captured once as a CUDA graph, and
// instances join or leave between cycles by rewriting the work lists only.
// An instance whose residual estimate has passed its tolerance skips the
// remaining steps of the cycle (per-instance step gate, as in the single
// instance solver).
//
// The server owns one device arena (its memory budget) and a worker thread:
// requests are admitted while a slot is free and the arena can hold the
// instance (coefficient tables, Krylov basis and work vectors), each cycle
// advances every resident instance, and finished instances are retired
// (solution copied to the host, memory returned) before the next cycle.
// Reductions are deterministic (per-chunk partials summed in a fixed order),
// so an instance's result does not depend on what else is in the batch.
//
// Precision: FP64, or FP32 operator inside FP64 iterative refinement -- the
// Arnoldi steps apply the FP32 operator, while each cycle ends with the true
// residual b - A x from the FP64 operator, so every restart is a refinement
// step and the stopping test is FP64.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>

#include "rt_device.cuh"

namespace rt {

namespace {

constexpr int kBT = 512;          // threads of the batched vector kernels
constexpr int kFormalWarps = 4;   // warps per CTA of the batched formal solver
constexpr int kInstThreads = 128; // threads of the per-instance scalar kernels
enum VecId { VX = 100, VB, VR, VW, VT, VTMP };

struct InstDev {
  int Ns, Nmu, Nnu, Nh, ngd, ngroups, fs, nchunks, chunk, m;
  int64_t nray, nd, N;
  int64_t cstride;   // columns of the FP64 tables (coef_col)
  int cshare;
  double xi, xiW2, inflow_bottom;
  const double *ce, *ca, *cb, *wnu, *wmu, *wray, *t201, *t202, *Minv;
  const float *dtau32, *r32, *wnu32, *wmu32, *t201f, *t202f;
  double *S, *S2;
  float* S32;
  double *V, *x, *b, *r, *w, *t, *tmp, *dinv, *part;
  GmresDev* gm;
};

struct InstStatus {
  double rel;
  double est;   // |g_{j+1}| / ||b|| of the instance's last Arnoldi step (rel before any)
  int iters, kstop, kdone, breakdown;
};

struct Counts {
  int nh, ng64, nc, ni;
  int ng32[3], off32[3];   // FP32 formal-solver items, grouped by formal solver
};

__device__ __forceinline__ double* vec(const InstDev& I, int id) {
  if (id < VX) return I.V + (int64_t)id * I.N;
  switch (id) {
    case VX: return I.x;
    case VB: return I.b;
    case VR: return I.r;
    case VW: return I.w;
    case VT: return I.t;
    default: return I.tmp;
  }
}

__device__ __forceinline__ bool step_gated(const InstDev& I, int step) {
  return step >= 0 && step >= I.gm->kstop;
}

__device__ __forceinline__ double bsum(double v) {
  __shared__ double red[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  __syncthreads();
  return s;
}

// an instance's partials: three buffers of kGramB sets of nchunks values
// (buffers 0 and 1 ping-pong between Arnoldi passes, buffer 2 holds the
// Gram dots of the newest basis vector)
__device__ __forceinline__ double* pset(const InstDev& I, int buf, int k) {
  return I.part + ((size_t)buf * kGramB + k) * I.nchunks;
}

// sqrt of the sum of an instance's chunk partials (set 0 of buffer pb, in a
// fixed order) and its inverse (0 for a zero norm), computed once by
// thread 0 (FP64 square roots and divisions are long FP64-pipe sequences)
__device__ __forceinline__ double inst_norm_inv(const InstDev& I, int pb, double* hn_out) {
  __shared__ double nb[2];
  if (threadIdx.x < 32) {
    double s = 0.0;
    for (int c = threadIdx.x; c < I.nchunks; c += 32) s += pset(I, pb, 0)[c];
    s = warp_sum(s);
    if (threadIdx.x == 0) {
      const double h = sqrt(s);
      nb[0] = h;
      nb[1] = h > 0.0 ? 1.0 / h : 0.0;
    }
  }
  __syncthreads();
  *hn_out = nb[0];
  const double inv = nb[1];
  __syncthreads();
  return inv;
}

// ------------------------------------------------------------ operator
// NORM (Arnoldi steps after the first): the input is v_src = w / ||w||, the
// last block pass's w scaled by the inverse norm kb_givens stored; it is
// written to v_src as the quadrature reads it, in place of a scaling pass
template <typename TC, int MODE, bool NORM = false>
__global__ void __launch_bounds__(kMomThreads) kb_moments(const InstDev* __restrict__ insts, const int2* __restrict__ wl,
                                                          const Counts* cnt, int src, int step, int useS2) {
  const int n = cnt->nh;
  for (int w = blockIdx.x; w < n; w += gridDim.x) {
    const int2 it = wl[w];
    const InstDev& I = insts[it.x];
    if (step_gated(I, step)) continue;
    const double* x = NORM ? I.w : vec(I, src);
    double* xo = NORM ? vec(I, src) : nullptr;
    const double inv = NORM ? I.gm->vscale : 1.0;
    if (sizeof(TC) == 8) {
      moments_flat64<MODE, false, NORM>(x, I.dinv, I.wray, I.t201, I.t202, I.Minv, I.Ns, I.Nmu, I.nray, I.xi,
                                        I.xiW2, useS2 ? I.S2 : I.S, it.y, inv, xo);
    } else {
      moments_height<double, float, MODE, NORM>(x, I.dinv, I.wnu32, I.wmu32, I.t201f, I.t202f, I.Minv, I.Ns, I.Nmu,
                                                I.Nnu, (float)I.xi, (float)I.xiW2, I.S32, it.y, inv, xo);
    }
    __syncthreads();
  }
}

template <typename TC, int FS, int MODE, int NS>
__device__ __forceinline__ void formal_item(const InstDev& I, int g, int s0, int src, int dst) {
  const int lane = threadIdx.x & 31;
  FormalArgs A;
  A.x = vec(I, src);
  A.dinv = I.dinv;
  A.ce = I.ce;
  A.ca = I.ca;
  A.cb = I.cb;
  A.cg = nullptr;
  A.cstride = I.cstride;
  A.cshare = I.cshare;
  A.dtau32 = I.dtau32;
  A.r32 = I.r32;
  A.S = sizeof(TC) == 8 ? (const void*)I.S : (const void*)I.S32;
  A.y = vec(I, dst);
  A.Ns = I.Ns;
  A.Nmu = I.Nmu;
  A.Nnu = I.Nnu;
  A.nray = I.nray;
  A.nd = I.nd;
  A.ngd = I.ngd;
  A.ntile = 1;
  A.inflow_bottom = I.inflow_bottom;
  A.kstop = nullptr;
  A.step = 0;
  const bool down = g < I.ngd;
  const int64_t base = down ? (int64_t)g * 32 : I.nd + (int64_t)(g - I.ngd) * 32;
  const int64_t end = down ? I.nd : I.nray;
  const bool active = base + lane < end;
  const int64_t r = active ? base + lane : end - 1;
  const int m = (int)(r / I.Nnu);
  const int Ns = I.Ns;
  TC Iv[NS];
#pragma unroll
  for (int q = 0; q < NS; ++q) Iv[q] = 0;
  if (active) {
    const int k0 = down ? 0 : Ns - 1;
    const double* x = reinterpret_cast<const double*>(A.x);
    double* y = reinterpret_cast<double*>(A.y);
#pragma unroll
    for (int q = 0; q < NS; ++q) {
      const int64_t o = (int64_t)(s0 + q) * Ns * I.nray + (int64_t)k0 * I.nray + r;
      if (MODE == KM_JACOBI) y[o] = x[o] * I.dinv[o];
      else y[o] = x[o];
    }
  }
  TC E = 1;
  if (sizeof(TC) == 8)
    sweep<TC, double, FS, MODE, 1, NS, kRing>(A, s0, down, r, m, active, 1, Ns, Iv, E);
  else
    sweep<TC, double, FS, MODE, 1, NS, kRing32>(A, s0, down, r, m, active, 1, Ns, Iv, E);
}

// FP64: items (slot, group, Stokes); FP32: items (slot, group) with both
// Stokes parameters per lane, one launch per formal solver (FS)
template <typename TC, int FS, int MODE>
__global__ void __launch_bounds__(32 * kFormalWarps) kb_formal(const InstDev* __restrict__ insts,
                                                               const int4* __restrict__ wl, const Counts* cnt,
                                                               int src, int dst, int step) {
  const int n = sizeof(TC) == 8 ? cnt->ng64 : cnt->ng32[FS];
  const int off = sizeof(TC) == 8 ? 0 : cnt->off32[FS];
  const int warps = gridDim.x * (blockDim.x >> 5);
  for (int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < n; w += warps) {
    const int4 it = wl[off + w];
    const InstDev& I = insts[it.x];
    if (step_gated(I, step)) continue;
    if (sizeof(TC) == 8) formal_item<TC, 0, MODE, 1>(I, it.y, it.z, src, dst);
    else formal_item<TC, FS, MODE, 2>(I, it.y, 0, src, dst);
  }
}

// ------------------------------------------------------------ vectors
#define CHUNK_LOOP(body)                                                      \
  {                                                                           \
    const int64_t lo = (int64_t)it.y * I.chunk;                               \
    const int64_t hi = lo + I.chunk < I.N ? lo + I.chunk : I.N;               \
    for (int64_t n_ = lo + threadIdx.x; n_ < hi; n_ += blockDim.x) { body }   \
  }

// Block MGS (the single-instance GMRES's Arnoldi step, per instance): passes
// of kGramB basis vectors, the MGS coefficients of a block from the dots r_k
// taken before it and the Gram entries, h_k = r_k - sum_{l<k} h_l <v_l, v_k>.

// warps k < n each sum set k of buffer buf into out[k] (fixed order)
__device__ __forceinline__ void inst_sets(const InstDev& I, int buf, int n, double* out) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp < n) {
    const double* p = pset(I, buf, warp);
    double s = 0.0;
    for (int c = lane; c < I.nchunks; c += 32) s += p[c];
    s = warp_sum(s);
    if (lane == 0) out[warp] = s;
  }
  __syncthreads();
}

// block sums of s[0..kGramB-1] (fixed order) for one chunk: sum k < n goes
// to set k of the instance's buffer buf, entry chunk
__device__ __forceinline__ void chunk_sum4(const double* s, int n, const InstDev& I, int buf, int chunk) {
  constexpr int NW = kBT / 32;
  static_assert(kGramB == 4 && kGramB * NW <= 64 && (NW & (NW - 1)) == 0, "reduction layout");
  __shared__ double red[kGramB][NW];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const double t = warp_sum4(s);
  if ((lane & 7) == 0) red[lane >> 3][warp] = t;
  __syncthreads();
  if (threadIdx.x < kGramB * NW) {
    const int k = threadIdx.x / NW, src = threadIdx.x % NW;
    double x = red[k][src];
#pragma unroll
    for (int o = NW / 2; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (src == 0 && k < n) pset(I, buf, k)[chunk] = x;
  }
  __syncthreads();
}

// The block sizes are template parameters: a DFMA under a false predicate
// still takes its FP64-pipe slot.

// first kernel of Arnoldi step j: partial dots <w, v_k>, k < NK, into buffer 0
template <int NK>
__global__ void __launch_bounds__(kBT) kb_bdot(const InstDev* __restrict__ insts, const int2* __restrict__ wl,
                                               const Counts* cnt, int j) {
  constexpr int nk = NK;
  for (int w = blockIdx.x; w < cnt->nc; w += gridDim.x) {
    const int2 it = wl[w];
    const InstDev& I = insts[it.x];
    if (step_gated(I, j)) continue;
    double s[kGramB] = {0.0, 0.0, 0.0, 0.0};
    CHUNK_LOOP(const double wi = I.w[n_]; double vv[kGramB]; _Pragma("unroll")
               for (int k = 0; k < kGramB; ++k) if (k < nk) vv[k] = I.V[(int64_t)k * I.N + n_]; _Pragma("unroll")
               for (int k = 0; k < kGramB; ++k) if (k < nk) s[k] = fma(wi, vv[k], s[k]);)
    chunk_sum4(s, nk, I, 0, it.y);
  }
}

// one block pass over v_{i0} .. v_{i0+NB-1} into buffer pb ^ 1: the dots with
// the next NN vectors, or, for the last block (NN == 0), ||w||^2 (set 0) and
// the Gram dots <w, v_{i0+k}>, k < ng (set 1+k; ng = NB when v_{j+1} shares
// the block, else 0)
template <int NB, int NN>
__global__ void __launch_bounds__(kBT) kb_bmgs(const InstDev* __restrict__ insts, const int2* __restrict__ wl,
                                               const Counts* cnt, int j, int i0, int pb) {
  static_assert(NB >= 1 && NB <= kGramB && NN >= 0 && NN <= kGramB && (NN == 0 || NB == kGramB), "block shape");
  constexpr int nb = NB, nn = NN, ng = NN == 0 && NB < kGramB ? NB : 0;
  __shared__ double rs[kGramB], hs[kGramB];
  for (int w = blockIdx.x; w < cnt->nc; w += gridDim.x) {
    const int2 it = wl[w];
    const InstDev& I = insts[it.x];
    if (step_gated(I, j)) continue;
    inst_sets(I, pb, nb, rs);
    if (threadIdx.x == 0) {
      for (int k = 0; k < nb; ++k) {
        double h = rs[k];
        for (int l = 0; l < k; ++l) h -= hs[l] * I.gm->gram[(i0 + k) * kGramB + (k - l)];
        hs[k] = h;
        if (it.y == 0) I.gm->H[j * (I.m + 1) + i0 + k] = h;
      }
    }
    __syncthreads();
    double h[kGramB];
#pragma unroll
    for (int k = 0; k < kGramB; ++k) h[k] = k < nb ? hs[k] : 0.0;
    __syncthreads();
    const double* vb = I.V + (int64_t)i0 * I.N;
    const double* vn = I.V + (int64_t)(i0 + nb) * I.N;
    double s[kGramB] = {0.0, 0.0, 0.0, 0.0};
    CHUNK_LOOP(double wi = I.w[n_]; double bv[kGramB]; _Pragma("unroll")
               for (int k = 0; k < kGramB; ++k) if (k < nb) bv[k] = vb[(int64_t)k * I.N + n_]; _Pragma("unroll")
               for (int k = 0; k < kGramB; ++k) if (k < nb) wi = fma(-h[k], bv[k], wi);
               I.w[n_] = wi;
               if constexpr (nn > 0) { _Pragma("unroll")
                 for (int k = 0; k < kGramB; ++k) if (k < nn) s[k] = fma(wi, vn[(int64_t)k * I.N + n_], s[k]);
               } else {
                 s[0] = fma(wi, wi, s[0]); _Pragma("unroll")
                 for (int k = 0; k < kGramB - 1; ++k) if (k < ng) s[1 + k] = fma(wi, bv[k], s[1 + k]);
               })
    chunk_sum4(s, nn ? nn : 1 + ng, I, pb ^ 1, it.y);
  }
}

// per instance: h_{j+1,j} = ||w|| and the Gram row j+1 of v_{j+1} from the
// last pass's partials (buffer pb, ng Gram sets), then the Givens rotations
// of column j and the residual estimate
__global__ void kb_givens(const InstDev* __restrict__ insts, const int* __restrict__ wi, const Counts* cnt, int j,
                          int pb, int ng) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= cnt->ni) return;
  const InstDev& I = insts[wi[q]];
  GmresDev* gm = I.gm;
  if (j >= gm->kstop) return;
  const int m = I.m;
  double* Hc = gm->H + j * (m + 1);
  double sets[kGramB] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int k = 0; k < kGramB; ++k) {
    if (k <= ng) {
      const double* p = pset(I, pb, k);
      double t = 0.0;
      for (int c = 0; c < I.nchunks; ++c) t += p[c];
      sets[k] = t;
    }
  }
  const double hj = sqrt(sets[0]);
  const double inv = hj > 0.0 ? 1.0 / hj : 0.0;
  Hc[j + 1] = hj;
  gm->vscale = inv;
#pragma unroll
  for (int k = 0; k < kGramB - 1; ++k)   // set 1+k: <w, v_{j+1-d}> with d = ng - k
    if (k < ng) gm->gram[(j + 1) * kGramB + (ng - k)] = sets[1 + k] * inv;
  for (int i = 0; i < j; ++i) {
    const double t = gm->cs[i] * Hc[i] + gm->sn[i] * Hc[i + 1];
    Hc[i + 1] = -gm->sn[i] * Hc[i] + gm->cs[i] * Hc[i + 1];
    Hc[i] = t;
  }
  const double a = Hc[j], b = Hc[j + 1];
  const double hn = hypot(a, b);
  if (hn == 0.0) {
    gm->breakdown = 1;
    gm->kstop = j;
    return;
  }
  const double c = a / hn, s = b / hn;
  gm->cs[j] = c;
  gm->sn[j] = s;
  Hc[j] = hn;
  Hc[j + 1] = 0.0;
  gm->g[j + 1] = -s * gm->g[j];
  gm->g[j] = c * gm->g[j];
  gm->iters += 1;
  gm->kdone = j + 1;
  const double est = fabs(gm->g[j + 1]) / gm->bnorm;
  gm->est = est;
  if (!(est >= gm->tol) || gm->iters >= gm->maxit || b == 0.0) gm->kstop = j + 1;
}

using KbBdotFn = void (*)(const InstDev*, const int2*, const Counts*, int);
using KbBmgsFn = void (*)(const InstDev*, const int2*, const Counts*, int, int, int);
static_assert(kGramB == 4, "kernel tables");
const KbBdotFn kb_bdot_fn[kGramB] = {kb_bdot<1>, kb_bdot<2>, kb_bdot<3>, kb_bdot<4>};
const KbBmgsFn kb_pass_fn[kGramB] = {kb_bmgs<4, 1>, kb_bmgs<4, 2>, kb_bmgs<4, 3>, kb_bmgs<4, 4>};
const KbBmgsFn kb_last_fn[kGramB] = {kb_bmgs<1, 0>, kb_bmgs<2, 0>, kb_bmgs<3, 0>, kb_bmgs<4, 0>};

__global__ void kb_lsq(const InstDev* __restrict__ insts, const int* __restrict__ wi, const Counts* cnt) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= cnt->ni) return;
  const InstDev& I = insts[wi[q]];
  GmresDev* gm = I.gm;
  const int k = gm->kdone, m = I.m;
  for (int i = k - 1; i >= 0; --i) {
    double s = gm->g[i];
    for (int l = i + 1; l < k; ++l) s -= gm->H[l * (m + 1) + i] * gm->y[l];
    gm->y[i] = s / gm->H[i * (m + 1) + i];
  }
}

// s = sum_{i<kdone} y_i V_i; mode 0: x += s, 1: x += dinv s, 2: t = s
__global__ void __launch_bounds__(kBT) kb_combine(const InstDev* __restrict__ insts, const int2* __restrict__ wl,
                                                  const Counts* cnt, int mode) {
  __shared__ double ys[kMaxRestart];
  for (int w = blockIdx.x; w < cnt->nc; w += gridDim.x) {
    const int2 it = wl[w];
    const InstDev& I = insts[it.x];
    const int k = I.gm->kdone;
    for (int i = threadIdx.x; i < k; i += blockDim.x) ys[i] = I.gm->y[i];
    __syncthreads();
    CHUNK_LOOP(double s = 0.0; for (int i = 0; i < k; ++i) s = fma(ys[i], I.V[(int64_t)i * I.N + n_], s);
               if (mode == 0) I.x[n_] += s; else if (mode == 1) I.x[n_] = fma(I.dinv[n_], s, I.x[n_]);
               else I.t[n_] = s;)
    __syncthreads();
  }
}

// x += t + beta* S2 (P^{-1} t with S2 = T M^{-1} J t)
__global__ void __launch_bounds__(kBT) kb_add_local(const InstDev* __restrict__ insts, const int2* __restrict__ wl,
                                                    const Counts* cnt) {
  for (int w = blockIdx.x; w < cnt->nc; w += gridDim.x) {
    const int2 it = wl[w];
    const InstDev& I = insts[it.x];
    CHUNK_LOOP(const int64_t rr = n_ % I.nray; const int64_t sk = n_ / I.nray; const int k = (int)(sk % I.Ns);
               const int s = (int)(sk / I.Ns); const int m = (int)(rr / I.Nnu);
               I.x[n_] += I.t[n_] + beta_star(I.cb, k, m, coef_col(rr, I.Nh, I.Nnu, I.cshare), I.cstride, I.Ns,
                                              I.Nh) *
                                         I.S2[((int64_t)s * I.Ns + k) * I.Nmu + m];)
  }
}

// r = b - tmp; partial ||r||^2 into part[0]
__global__ void __launch_bounds__(kBT) kb_residual(const InstDev* __restrict__ insts, const int2* __restrict__ wl,
                                                   const Counts* cnt) {
  for (int w = blockIdx.x; w < cnt->nc; w += gridDim.x) {
    const int2 it = wl[w];
    const InstDev& I = insts[it.x];
    double s = 0.0;
    CHUNK_LOOP(const double v = I.b[n_] - I.tmp[n_]; I.r[n_] = v; s = fma(v, v, s);)
    s = bsum(s);
    if (threadIdx.x == 0) I.part[it.y] = s;
  }
}

__global__ void kb_set_bnorm(const InstDev* __restrict__ insts, const int* __restrict__ wi, const Counts* cnt) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= cnt->ni) return;
  const InstDev& I = insts[wi[q]];
  double s = 0.0;
  for (int c = 0; c < I.nchunks; ++c) s += I.part[c];
  I.gm->bnorm = sqrt(s);
}

// start of a cycle: beta = ||r||, v_0 = r / beta, g = beta e_1, step budget
__global__ void __launch_bounds__(kBT) kb_cycle_start(const InstDev* __restrict__ insts, const int2* __restrict__ wl,
                                                      const Counts* cnt, InstStatus* __restrict__ status) {
  for (int w = blockIdx.x; w < cnt->nc; w += gridDim.x) {
    const int2 it = wl[w];
    const InstDev& I = insts[it.x];
    double rn;
    const double inv = inst_norm_inv(I, 0, &rn);
    CHUNK_LOOP(I.V[n_] = I.r[n_] * inv;)
    if (it.y == 0 && threadIdx.x == 0) {
      GmresDev* gm = I.gm;
      gm->rnorm = rn;
      gm->rel = gm->bnorm > 0.0 ? rn / gm->bnorm : 0.0;
      for (int i = 0; i <= I.m; ++i) gm->g[i] = 0.0;
      gm->g[0] = rn;
      gm->kdone = 0;
      const int left = gm->maxit - gm->iters;
      gm->kstop = left < I.m ? (left > 0 ? left : 0) : I.m;
      if (!(gm->rel >= gm->tol)) gm->kstop = 0;
      InstStatus st;
      st.rel = gm->rel;
      st.est = gm->iters > 0 ? gm->est : gm->rel;
      st.iters = gm->iters;
      st.kstop = gm->kstop;
      st.kdone = gm->kdone;
      st.breakdown = gm->breakdown;
      status[it.x] = st;
    }
  }
}

#undef CHUNK_LOOP

// ------------------------------------------------------------ arena
// First-fit allocator over one device allocation (256-byte granules).
class Arena : public DevAllocator {
 public:
  // one block of `bytes` from src (NULL: cudaMalloc)
  rt_status init(size_t bytes, DevAllocator* src) {
    bytes_ = (bytes + 255) & ~(size_t)255;
    src_ = src;
    cudaError_t e = src ? src->alloc(&base_, bytes_) : cudaMalloc(&base_, bytes_);
    if (e != cudaSuccess) {
      set_error("arena allocation of %zu bytes failed: %s", bytes_, cudaGetErrorString(e));
      base_ = nullptr;
      return RT_ENOMEM;
    }
    free_[0] = bytes_;
    return RT_OK;
  }
  // gives the block back to its source (before the source goes away)
  void teardown() {
    if (base_) {
      if (src_) src_->release(base_);
      else cudaFree(base_);
    }
    base_ = nullptr;
  }
  ~Arena() override { teardown(); }
  cudaError_t alloc(void** p, size_t bytes) override {
    std::lock_guard<std::mutex> lk(mu_);
    bytes = (bytes + 255) & ~(size_t)255;
    if (bytes == 0) bytes = 256;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        const size_t off = it->first, len = it->second;
        free_.erase(it);
        if (len > bytes) free_[off + bytes] = len - bytes;
        used_[off] = bytes;
        *p = static_cast<char*>(base_) + off;
        in_use_ += bytes;
        return cudaSuccess;
      }
    }
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  void release(void* p) override {
    if (!p) return;
    std::lock_guard<std::mutex> lk(mu_);
    const size_t off = static_cast<char*>(p) - static_cast<char*>(base_);
    auto u = used_.find(off);
    if (u == used_.end()) return;
    size_t len = u->second;
    used_.erase(u);
    in_use_ -= len;
    size_t start = off;
    auto nx = free_.lower_bound(off);
    if (nx != free_.end() && nx->first == off + len) {   // merge with the next hole
      len += nx->second;
      free_.erase(nx);
    }
    auto pv = free_.lower_bound(off);
    if (pv != free_.begin()) {                           // merge with the previous hole
      --pv;
      if (pv->first + pv->second == off) {
        start = pv->first;
        len += pv->second;
        free_.erase(pv);
      }
    }
    free_[start] = len;
  }
  size_t largest_hole() {
    std::lock_guard<std::mutex> lk(mu_);
    size_t b = 0;
    for (auto& kv : free_) b = std::max(b, kv.second);
    return b;
  }
  size_t in_use() {
    std::lock_guard<std::mutex> lk(mu_);
    return in_use_;
  }

 private:
  void* base_ = nullptr;
  DevAllocator* src_ = nullptr;
  size_t bytes_ = 0, in_use_ = 0;
  std::map<size_t, size_t> free_, used_;
  std::mutex mu_;
};

inline double wall_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

// ------------------------------------------------------------ host side
struct Request {
  uint64_t ticket = 0;
  rt_problem_desc desc{};
  std::vector<double> tau, B, phi;
  double rtol = 1e-8;
  int maxit = 10000;
  double t_submit = 0, t_done = 0;
  std::vector<double> x;   // solution on completion
  rt_solve_info info{};
  bool done = false;
  double deadline = 0;             // wall time (ms) past which the request is cancelled; 0: none
  std::atomic<bool> cancel{false}; // set by rt_batch_cancel for a resident request
};

struct Instance {
  Request* req = nullptr;
  Problem P;
  int slot = -1;
  int cycles = 0;
  InstDev dev{};
  void* block = nullptr;   // solver buffers (one arena block)
};

struct Server {
  rt_server_opts opts{};
  int device = 0, sms = 0;
  DevAllocator* hook = nullptr;   // the caller's allocator (owned), or NULL for cudaMalloc
  Arena arena;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request*> pending;
  std::map<uint64_t, std::unique_ptr<Request>> requests;
  std::atomic<uint64_t> next_ticket{1};
  std::thread worker;
  bool stop = false;
  std::string worker_error;
  rt_status worker_status = RT_OK;
  // worker-owned state
  cudaStream_t st = nullptr, cap = nullptr;
  std::vector<Instance*> slots;   // index = slot
  InstDev* d_insts = nullptr;
  InstStatus* d_status = nullptr;
  Counts* d_counts = nullptr;
  int2 *d_wl_h = nullptr, *d_wl_c = nullptr;
  int4 *d_wl_g64 = nullptr, *d_wl_g32 = nullptr;
  int* d_wl_i = nullptr;
  size_t cap_h = 0, cap_c = 0, cap_g64 = 0, cap_g32 = 0;
  int2* d_wl_new_c = nullptr;   // admission work lists (new instances only)
  int* d_wl_new_i = nullptr;
  Counts* d_new_counts = nullptr;
  size_t cap_new_c = 0;
  cudaGraphExec_t graph = nullptr;
  long long graph_kernels = 0;
  std::atomic<long long> cycles{0}, completed{0};
  std::atomic<int> resident{0};
  int grid_h = 0, grid_g = 0, grid_v = 0, grid_i = 0;   // persistent grids (CTAs)
  bool tuned = false;                                    // autotune_grids has run
  int tuned_at = 0;                                      // resident instances at the tuning
};

namespace {

// the server's own device buffers: from the caller's allocator when given
cudaError_t srv_alloc(Server* S, void** p, size_t bytes) {
  const cudaError_t e = S->hook ? S->hook->alloc(p, bytes) : cudaMalloc(p, bytes);
  return e == cudaSuccess ? poison_fill(*p, bytes) : e;
}
void srv_free(Server* S, void* p) {
  if (!p) return;
  if (S->hook) S->hook->release(p);
  else cudaFree(p);
}

template <typename T>
rt_status grow(Server* S, T** p, size_t* cap, size_t need) {
  if (need <= *cap) return RT_OK;
  if (*p) {
    // the previous cycle's kernels may still read the old list
    RT_TRY_CUDA(cudaStreamSynchronize(S->st));
    srv_free(S, *p);
  }
  *p = nullptr;
  *cap = 0;
  size_t c = need + need / 2 + 64;
  RT_TRY_CUDA(srv_alloc(S, (void**)p, c * sizeof(T)));
  *cap = c;
  return RT_OK;
}

// instance footprint of the solver buffers: basis (m+1), six work vectors,
// the Jacobi inverse diagonal, partials, GMRES state
size_t solver_bytes(int64_t N, int m, int nchunks) {
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  return al((size_t)(m + 1) * N * 8) + 7 * al((size_t)N * 8) + al((size_t)3 * kGramB * nchunks * 8) +
         al(sizeof(GmresDev));
}

int64_t chunk_for(int64_t N) {
  (void)N;
  return 65536;
}

template <int MODE>
void formal32(Server* S, cudaStream_t st, int src, int dst, int step) {
  kb_formal<float, RT_FS_DELO_LINEAR, MODE><<<S->grid_g, 32 * kFormalWarps, 0, st>>>(S->d_insts, S->d_wl_g32,
                                                                                     S->d_counts, src, dst, step); RT_COUNT(1);
  kb_formal<float, RT_FS_IMPLICIT_EULER, MODE><<<S->grid_g, 32 * kFormalWarps, 0, st>>>(S->d_insts, S->d_wl_g32,
                                                                                        S->d_counts, src, dst, step); RT_COUNT(1);
  kb_formal<float, RT_FS_TRAPEZOIDAL, MODE><<<S->grid_g, 32 * kFormalWarps, 0, st>>>(S->d_insts, S->d_wl_g32,
                                                                                     S->d_counts, src, dst, step); RT_COUNT(1);
}

template <bool NORM>
void enqueue_apply_t(Server* S, cudaStream_t st, int src, int dst, int md, bool f32, int step) {
  const InstDev* I = S->d_insts;
  const Counts* C = S->d_counts;
  if (!f32) {
    switch (md) {
      case KM_JACOBI:
        kb_moments<double, KM_JACOBI, NORM><<<S->grid_h, kMomThreads, 0, st>>>(I, S->d_wl_h, C, src, step, 0); RT_COUNT(1);
        kb_formal<double, 0, KM_JACOBI><<<S->grid_g, 32 * kFormalWarps, 0, st>>>(I, S->d_wl_g64, C, src, dst, step); RT_COUNT(1);
        break;
      case KM_LOCAL_LAMBDA:
        kb_moments<double, KM_LOCAL_LAMBDA, NORM><<<S->grid_h, kMomThreads, 0, st>>>(I, S->d_wl_h, C, src, step, 0); RT_COUNT(1);
        kb_formal<double, 0, KM_LOCAL_LAMBDA><<<S->grid_g, 32 * kFormalWarps, 0, st>>>(I, S->d_wl_g64, C, src, dst,
                                                                                     step); RT_COUNT(1);
        break;
      default:
        kb_moments<double, KM_PLAIN, NORM><<<S->grid_h, kMomThreads, 0, st>>>(I, S->d_wl_h, C, src, step, 0); RT_COUNT(1);
        kb_formal<double, 0, KM_PLAIN><<<S->grid_g, 32 * kFormalWarps, 0, st>>>(I, S->d_wl_g64, C, src, dst, step); RT_COUNT(1);
    }
  } else {
    switch (md) {
      case KM_JACOBI:
        kb_moments<float, KM_JACOBI, NORM><<<S->grid_h, kMomThreads, 0, st>>>(I, S->d_wl_h, C, src, step, 0); RT_COUNT(1);
        formal32<KM_JACOBI>(S, st, src, dst, step);
        break;
      case KM_LOCAL_LAMBDA:
        kb_moments<float, KM_LOCAL_LAMBDA, NORM><<<S->grid_h, kMomThreads, 0, st>>>(I, S->d_wl_h, C, src, step, 0); RT_COUNT(1);
        formal32<KM_LOCAL_LAMBDA>(S, st, src, dst, step);
        break;
      default:
        kb_moments<float, KM_PLAIN, NORM><<<S->grid_h, kMomThreads, 0, st>>>(I, S->d_wl_h, C, src, step, 0); RT_COUNT(1);
        formal32<KM_PLAIN>(S, st, src, dst, step);
    }
  }
}

// the operator of every resident instance: w[dst] = A v[src] (quadrature,
// then the formal solver), with the server's current grids; norm: v[src] is
// first formed as w / ||w|| by the quadrature kernel (see kb_moments)
void enqueue_apply(Server* S, cudaStream_t st, int src, int dst, int md, bool f32, int step, bool norm = false) {
  if (norm) enqueue_apply_t<true>(S, st, src, dst, md, f32, step);
  else enqueue_apply_t<false>(S, st, src, dst, md, f32, step);
}

// Autotuner of the persistent grids: CTAs per SM of the quadrature, the
// formal-solver and the vector kernels.  Run once per server, when at least
// kTuneResident instances (or all slots) are resident, so the timing reflects
// a loaded batch rather than the first request of a stream; the cycle graph
// is recaptured with the result.  Every candidate
// pair of quadrature / formal-solver grids runs the operator of the first
// Arnoldi step, every vector grid a dot-product pass, twice each, timed
// with events on the worker's stream; the fastest are kept.  The probe writes
// only what the cycle recomputes before reading (the source functions, w,
// the partials of buffer 0), and the batch's reductions do not depend on the
// grid (one block per work item), so tuning changes no result.
constexpr int kTuneResident = 64;   // resident instances that make the timing representative
constexpr float kTuneMargin = 0.95f; // a candidate must beat the current grid by 5%

rt_status autotune_grids(Server* S, int resident) {
  const int prec = S->opts.precond;
  const bool fp32 = S->opts.precision == RT_PRECISION_FP32_REFINE;
  const int mode = prec == RT_PREC_JACOBI ? KM_JACOBI : prec == RT_PREC_LOCAL_LAMBDA ? KM_LOCAL_LAMBDA : KM_PLAIN;
  cudaStream_t st = S->st;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  RT_TRY_CUDA(cudaEventCreate(&e0));
  cudaError_t ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) {
    cudaEventDestroy(e0);
    RT_TRY_CUDA(ce);
  }
  auto timeit = [&](auto&& launch, float* ms) -> cudaError_t {
    launch();   // warm-up
    cudaError_t e = cudaEventRecord(e0, st);
    for (int r = 0; r < 2 && e == cudaSuccess; ++r) launch();
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    return e;
  };
  const int sms = S->sms;
  cudaError_t e = cudaSuccess;
  // one grid at a time (formal solver, quadrature, vector kernels), each
  // candidate against the current choice, which it must beat by kTuneMargin
  auto tune = [&](int* grid, const int (&per_sm)[3], auto&& launch) {
    const int keep = *grid;
    float best = 0.f;
    e = timeit(launch, &best);
    int pick = keep;
    for (int c : per_sm) {
      if (e != cudaSuccess || c * sms == keep) continue;
      *grid = c * sms;
      float ms = 0.f;
      e = timeit(launch, &ms);
      if (e == cudaSuccess && ms < kTuneMargin * best) {
        best = ms;
        pick = *grid;
      }
    }
    *grid = pick;
  };
  const int gs[] = {4, 8, 16}, hs[] = {2, 4, 8}, vs[] = {4, 8, 16};
  auto apply = [&] { enqueue_apply(S, st, 0, VW, mode, fp32, 0); RT_COUNT(fp32 ? 4 : 2); };
  tune(&S->grid_g, gs, apply);
  tune(&S->grid_h, hs, apply);
  // the vector grid on the kernel that dominates the cycle: a full block
  // pass (4 updates, 4 look-ahead dots) of Arnoldi step 7; it writes only
  // w, one partial buffer and rows 0-3 of Hessenberg column 7, all of which
  // step 7 of the cycle recomputes before reading them
  tune(&S->grid_v, vs, [&] {
    if (S->opts.restart >= 2 * kGramB)
      kb_pass_fn[kGramB - 1]<<<S->grid_v, kBT, 0, st>>>(S->d_insts, S->d_wl_c, S->d_counts, 2 * kGramB - 1, 0, 0);
    else
      kb_bdot<1><<<S->grid_v, kBT, 0, st>>>(S->d_insts, S->d_wl_c, S->d_counts, 0);
    RT_COUNT(1);
  });
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  S->tuned = true;
  S->tuned_at = resident;
  RT_TRY_CUDA(e);
  return RT_OK;
}

// enqueue one restart cycle for all resident instances (captured once)
rt_status enqueue_batch_cycle(Server* S, cudaStream_t st) {
  const int m = S->opts.restart;
  const int prec = S->opts.precond;
  const bool fp32 = S->opts.precision == RT_PRECISION_FP32_REFINE;
  const int mode = prec == RT_PREC_JACOBI ? KM_JACOBI : prec == RT_PREC_LOCAL_LAMBDA ? KM_LOCAL_LAMBDA : KM_PLAIN;
  const InstDev* I = S->d_insts;
  const Counts* C = S->d_counts;
  for (int j = 0; j < m; ++j) {
    // steps after the first normalise v_j = w / ||w|| inside the quadrature
    enqueue_apply(S, st, j, VW, mode, fp32, j, j > 0);
    int pb = 0;
    kb_bdot_fn[std::min(kGramB, j + 1) - 1]<<<S->grid_v, kBT, 0, st>>>(I, S->d_wl_c, C, j); RT_COUNT(1);
    for (int i0 = 0; i0 <= j; i0 += kGramB) {
      const int nb = std::min(kGramB, j + 1 - i0);
      const int nn = std::max(0, std::min(kGramB, j + 1 - (i0 + nb)));
      (nn ? kb_pass_fn[nn - 1] : kb_last_fn[nb - 1])<<<S->grid_v, kBT, 0, st>>>(I, S->d_wl_c, C, j, i0, pb); RT_COUNT(1);
      pb ^= 1;
    }
    // h_{j+1,j}, the Gram row, the rotations and the inverse norm that the
    // next step's quadrature scales w by; an instance that stops at step j
    // never forms v_{j+1}, which no later kernel of the cycle reads
    const int ng = (j + 1) % kGramB;
    kb_givens<<<S->grid_i, kInstThreads, 0, st>>>(I, S->d_wl_i, C, j, pb, ng); RT_COUNT(1);
  }
  kb_lsq<<<S->grid_i, kInstThreads, 0, st>>>(I, S->d_wl_i, C); RT_COUNT(1);
  if (mode == KM_LOCAL_LAMBDA) {
    kb_combine<<<S->grid_v, kBT, 0, st>>>(I, S->d_wl_c, C, 2); RT_COUNT(1);
    kb_moments<double, KM_LOCAL_LAMBDA><<<S->grid_h, kMomThreads, 0, st>>>(I, S->d_wl_h, C, VT, -1, 1); RT_COUNT(1);
    kb_add_local<<<S->grid_v, kBT, 0, st>>>(I, S->d_wl_c, C); RT_COUNT(1);
  } else {
    kb_combine<<<S->grid_v, kBT, 0, st>>>(I, S->d_wl_c, C, mode == KM_JACOBI ? 1 : 0); RT_COUNT(1);
  }
  enqueue_apply(S, st, VX, VTMP, KM_PLAIN, false, -1);   // FP64 true residual
  kb_residual<<<S->grid_v, kBT, 0, st>>>(I, S->d_wl_c, C); RT_COUNT(1);
  kb_cycle_start<<<S->grid_v, kBT, 0, st>>>(I, S->d_wl_c, C, S->d_status); RT_COUNT(1);
  RT_TRY_CUDA(cudaGetLastError());
  return RT_OK;
}

rt_status capture_cycle(Server* S) {
  if (S->graph) return RT_OK;
  RT_TRY_CUDA(cudaStreamBeginCapture(S->cap, cudaStreamCaptureModeThreadLocal));
  g_capturing = 1;
  rt_status s = enqueue_batch_cycle(S, S->cap);
  g_capturing = 0;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(S->cap, &g);
  if (s != RT_OK) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  if (e != cudaSuccess) {
    set_error("batch graph capture failed: %s", cudaGetErrorString(e));
    return RT_ECUDA;
  }
  size_t nn = 0;
  S->graph_kernels = 0;
  if (cudaGraphGetNodes(g, nullptr, &nn) == cudaSuccess && nn) {
    std::vector<cudaGraphNode_t> nodes(nn);
    if (cudaGraphGetNodes(g, nodes.data(), &nn) == cudaSuccess)
      for (size_t i = 0; i < nn; ++i) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++S->graph_kernels;
      }
  }
  e = cudaGraphInstantiate(&S->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    S->graph = nullptr;
    set_error("batch graph instantiate failed: %s", cudaGetErrorString(e));
    return RT_ECUDA;
  }
  return RT_OK;
}

void drop_graph(Server* S) {
  if (S->graph) cudaGraphExecDestroy(S->graph);
  S->graph = nullptr;
}

// rebuild the work lists of all resident instances
rt_status rebuild_lists(Server* S) {
  std::vector<int2> h, c;
  std::vector<int4> g64, g32, g32f[3];
  std::vector<int> wi;
  for (size_t q = 0; q < S->slots.size(); ++q) {
    Instance* in = S->slots[q];
    if (!in) continue;
    const int sl = (int)q;
    wi.push_back(sl);
    for (int k = 0; k < in->P.Ns; ++k) h.push_back(make_int2(sl, k));
    for (int g = 0; g < in->P.ngroups; ++g) {
      g32f[in->P.fs].push_back(make_int4(sl, g, 0, 0));
      for (int s = 0; s < 2; ++s) g64.push_back(make_int4(sl, g, s, 0));
    }
    for (int cc = 0; cc < in->dev.nchunks; ++cc) c.push_back(make_int2(sl, cc));
  }
  Counts cn{(int)h.size(), (int)g64.size(), (int)c.size(), (int)wi.size(), {0, 0, 0}, {0, 0, 0}};
  for (int f = 0; f < 3; ++f) {
    cn.off32[f] = (int)g32.size();
    cn.ng32[f] = (int)g32f[f].size();
    g32.insert(g32.end(), g32f[f].begin(), g32f[f].end());
  }
  // interleave the formal-solver items of different instances so that big
  // instances do not end up on the same SMs
  bool regrown = false;
  const size_t ch = S->cap_h, cc = S->cap_c, c64 = S->cap_g64, c32 = S->cap_g32;
  RT_TRY(grow(S, &S->d_wl_h, &S->cap_h, h.size()));
  RT_TRY(grow(S, &S->d_wl_c, &S->cap_c, c.size()));
  RT_TRY(grow(S, &S->d_wl_g64, &S->cap_g64, g64.size()));
  RT_TRY(grow(S, &S->d_wl_g32, &S->cap_g32, g32.size()));
  regrown = ch != S->cap_h || cc != S->cap_c || c64 != S->cap_g64 || c32 != S->cap_g32;
  if (regrown) drop_graph(S);
  if (!h.empty()) RT_TRY_CUDA(cudaMemcpyAsync(S->d_wl_h, h.data(), h.size() * sizeof(int2), cudaMemcpyHostToDevice, S->st));
  if (!c.empty()) RT_TRY_CUDA(cudaMemcpyAsync(S->d_wl_c, c.data(), c.size() * sizeof(int2), cudaMemcpyHostToDevice, S->st));
  if (!g64.empty())
    RT_TRY_CUDA(cudaMemcpyAsync(S->d_wl_g64, g64.data(), g64.size() * sizeof(int4), cudaMemcpyHostToDevice, S->st));
  if (!g32.empty())
    RT_TRY_CUDA(cudaMemcpyAsync(S->d_wl_g32, g32.data(), g32.size() * sizeof(int4), cudaMemcpyHostToDevice, S->st));
  if (!wi.empty()) RT_TRY_CUDA(cudaMemcpyAsync(S->d_wl_i, wi.data(), wi.size() * sizeof(int), cudaMemcpyHostToDevice, S->st));
  RT_TRY_CUDA(cudaMemcpyAsync(S->d_counts, &cn, sizeof cn, cudaMemcpyHostToDevice, S->st));
  RT_TRY_CUDA(cudaStreamSynchronize(S->st));
  return RT_OK;
}

void free_instance(Server* S, Instance* in) {
  if (in->block) S->arena.release(in->block);
  in->block = nullptr;
  free_device(&in->P);
}

// build one instance in the arena: tables, rhs, preconditioner data, solver buffers
rt_status make_instance(Server* S, Request* rq, Instance* in, int slot) {
  in->req = rq;
  in->slot = slot;
  Problem& P = in->P;
  P.alloc = &S->arena;
  P.in_arena = 1;
  host_grids(&rq->desc, P);
  P.device = S->device;
  P.num_sms = S->sms;
  RT_TRY(setup_device_tables(&P, S->st));
  const int m = S->opts.restart;
  const int64_t N = P.N;
  const int64_t chunk = chunk_for(N);
  const int nchunks = (int)((N + chunk - 1) / chunk);
  const size_t bytes = solver_bytes(N, m, nchunks);
  void* blk = nullptr;
  if (S->arena.alloc(&blk, bytes) != cudaSuccess) {
    set_error("arena full");
    return RT_ENOMEM;
  }
  in->block = blk;
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  char* p = static_cast<char*>(blk);
  InstDev& D = in->dev;
  D.V = reinterpret_cast<double*>(p);
  p += al((size_t)(m + 1) * N * 8);
  double** vecs[] = {&D.x, &D.b, &D.r, &D.w, &D.t, &D.tmp, &D.dinv};
  for (double** v : vecs) {
    *v = reinterpret_cast<double*>(p);
    p += al((size_t)N * 8);
  }
  D.part = reinterpret_cast<double*>(p);
  p += al((size_t)3 * kGramB * nchunks * 8);
  D.gm = reinterpret_cast<GmresDev*>(p);
  D.Ns = P.Ns;
  D.Nmu = P.Nmu;
  D.Nnu = P.Nnu;
  D.Nh = P.Nh;
  D.ngd = P.ngroups / 2;
  D.ngroups = P.ngroups;
  D.fs = P.fs;
  D.nchunks = nchunks;
  D.chunk = (int)chunk;
  D.m = m;
  D.nray = P.nray;
  D.nd = P.nd;
  D.N = N;
  D.xi = P.xi;
  D.xiW2 = P.xi * P.W2;
  D.inflow_bottom = P.B[P.Ns - 1];
  D.ce = P.ce;
  D.ca = P.ca;
  D.cb = P.cb;
  D.cstride = P.cstride;
  D.cshare = P.cshare;
  D.wnu = P.wI2;
  D.wmu = P.wQ2;
  D.wray = P.wray;
  D.t201 = P.t201d;
  D.t202 = P.t202d;
  D.Minv = P.Minv;
  D.dtau32 = P.dtau32;
  D.r32 = P.r32;
  D.wnu32 = P.wI2f;
  D.wmu32 = P.wQ2f;
  D.t201f = P.t201f;
  D.t202f = P.t202f;
  D.S = P.S;
  D.S2 = P.S2;
  D.S32 = P.S32;
  // rhs, preconditioner, x0 = 0, GMRES state
  P.dinv = D.dinv;
  RT_TRY(op_rhs(&P, D.b, S->st));
  if (S->opts.precond == RT_PREC_JACOBI) RT_TRY(op_jacobi_inv(&P, D.dinv, S->st));
  P.dinv = nullptr;   // the arena block owns it
  RT_TRY_CUDA(cudaMemsetAsync(D.x, 0, (size_t)N * 8, S->st));
  RT_TRY_CUDA(cudaMemsetAsync(D.tmp, 0, (size_t)N * 8, S->st));
  std::unique_ptr<GmresDev> initp(new GmresDev);   // large arrays: not on the stack
  GmresDev& init = *initp;
  memset(&init, 0, kGmresHeader);
  init.tol = rq->rtol;
  init.maxit = rq->maxit;
  RT_TRY_CUDA(cudaMemcpyAsync(D.gm, &init, kGmresHeader, cudaMemcpyHostToDevice, S->st));
  RT_TRY_CUDA(cudaMemcpyAsync(S->d_insts + slot, &D, sizeof D, cudaMemcpyHostToDevice, S->st));
  RT_TRY_CUDA(cudaStreamSynchronize(S->st));   // init is freed on return
  return RT_OK;
}

// prologue of newly admitted instances: r = b, ||b||, v_0, step budget
rt_status start_instances(Server* S, const std::vector<Instance*>& fresh) {
  std::vector<int2> c;
  std::vector<int> wi;
  for (Instance* in : fresh) {
    wi.push_back(in->slot);
    for (int cc = 0; cc < in->dev.nchunks; ++cc) c.push_back(make_int2(in->slot, cc));
  }
  RT_TRY(grow(S, &S->d_wl_new_c, &S->cap_new_c, c.size()));
  RT_TRY_CUDA(cudaMemcpyAsync(S->d_wl_new_c, c.data(), c.size() * sizeof(int2), cudaMemcpyHostToDevice, S->st));
  RT_TRY_CUDA(cudaMemcpyAsync(S->d_wl_new_i, wi.data(), wi.size() * sizeof(int), cudaMemcpyHostToDevice, S->st));
  Counts cn{0, 0, (int)c.size(), (int)wi.size(), {0, 0, 0}, {0, 0, 0}};
  RT_TRY_CUDA(cudaMemcpyAsync(S->d_new_counts, &cn, sizeof cn, cudaMemcpyHostToDevice, S->st));
  kb_residual<<<S->grid_v, kBT, 0, S->st>>>(S->d_insts, S->d_wl_new_c, S->d_new_counts); RT_COUNT(1);
  kb_set_bnorm<<<(int)((wi.size() + kInstThreads - 1) / kInstThreads), kInstThreads, 0, S->st>>>(
      S->d_insts, S->d_wl_new_i, S->d_new_counts); RT_COUNT(1);
  kb_cycle_start<<<S->grid_v, kBT, 0, S->st>>>(S->d_insts, S->d_wl_new_c, S->d_new_counts, S->d_status); RT_COUNT(1);
  RT_TRY_CUDA(cudaGetLastError());
  return RT_OK;
}

void finish_request(Server* S, Instance* in, const InstStatus& st, rt_status status) {
  Request* rq = in->req;
  rq->x.resize(in->P.N);
  cudaMemcpyAsync(rq->x.data(), in->dev.x, (size_t)in->P.N * 8, cudaMemcpyDeviceToHost, S->st);
  cudaStreamSynchronize(S->st);
  rq->info.status = status;
  rq->info.iters = st.iters;
  rq->info.restarts = in->cycles;
  rq->info.applies = st.iters + in->cycles;
  rq->info.refine_steps = S->opts.precision == RT_PRECISION_FP32_REFINE ? in->cycles : 0;
  rq->info.rel_resid = st.rel;
  rq->info.err_est = st.est;
  rq->t_done = wall_ms();
  rq->info.t_total_ms = rq->t_done - rq->t_submit;
  std::lock_guard<std::mutex> lk(S->mu);
  rq->done = true;
  S->completed.fetch_add(1);
}

void worker_main(Server* S) {
  cudaSetDevice(S->device);
  auto fail = [&](rt_status s) {
    std::lock_guard<std::mutex> lk(S->mu);
    S->worker_status = s;
    S->worker_error = rt_last_error();
    for (Request* rq : S->pending) {
      rq->info.status = s;
      rq->done = true;
    }
    S->pending.clear();
    for (Instance* in : S->slots)
      if (in) {
        in->req->info.status = s;
        in->req->done = true;
      }
  };
  std::vector<InstStatus> hs;
  for (;;) {
    // admission
    std::vector<Request*> admit;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      bool any_active = false;
      for (Instance* in : S->slots) any_active |= in != nullptr;
      if (!any_active) S->cv.wait(lk, [&] { return S->stop || !S->pending.empty(); });
      if (S->stop) break;
      // queued requests past their deadline (anywhere in the queue) end unadmitted
      const double now = wall_ms();
      for (auto q = S->pending.begin(); q != S->pending.end();) {
        Request* rq = *q;
        if (rq->cancel.load() || (rq->deadline > 0.0 && now > rq->deadline)) {
          rq->info.status = RT_ECANCELED;
          rq->t_done = now;
          rq->info.t_total_ms = rq->t_done - rq->t_submit;
          rq->done = true;
          S->completed.fetch_add(1);
          q = S->pending.erase(q);
        } else {
          ++q;
        }
      }
      int freeslots = 0;
      for (Instance* in : S->slots) freeslots += in == nullptr;
      while (!S->pending.empty() && (int)admit.size() < freeslots) {
        admit.push_back(S->pending.front());
        S->pending.pop_front();
      }
    }
    std::vector<Instance*> fresh;
    std::vector<Request*> back;   // did not fit: requeue at the front
    for (Request* rq : admit) {
      int slot = -1;
      for (size_t q = 0; q < S->slots.size(); ++q)
        if (!S->slots[q]) {
          slot = (int)q;
          break;
        }
      Instance* in = new Instance();
      rt_status s = make_instance(S, rq, in, slot);
      if (s == RT_ENOMEM) {
        free_instance(S, in);
        delete in;
        back.push_back(rq);
        continue;
      }
      if (s != RT_OK) {
        free_instance(S, in);
        delete in;
        std::lock_guard<std::mutex> lk(S->mu);
        rq->info.status = s;
        rq->done = true;
        S->completed.fetch_add(1);
        continue;
      }
      S->slots[slot] = in;
      fresh.push_back(in);
      S->resident.fetch_add(1);
    }
    if (!back.empty()) {
      std::lock_guard<std::mutex> lk(S->mu);
      for (auto it = back.rbegin(); it != back.rend(); ++it) S->pending.push_front(*it);
    }
    bool any = false;
    for (Instance* in : S->slots) any |= in != nullptr;
    if (!any) {
      if (!back.empty()) {
        // the arena cannot hold even one of them alone: fail the head request
        std::lock_guard<std::mutex> lk(S->mu);
        Request* rq = S->pending.front();
        S->pending.pop_front();
        rq->info.status = RT_ENOMEM;
        rq->done = true;
        S->completed.fetch_add(1);
      }
      continue;
    }
    rt_status s = RT_OK;
    if (!fresh.empty()) s = start_instances(S, fresh);
    if (s == RT_OK) s = rebuild_lists(S);
    if (s == RT_OK && S->opts.autotune && !S->tuned) {
      int nres = 0;
      for (Instance* in : S->slots) nres += in != nullptr;
      if (nres >= std::min(kTuneResident, S->opts.max_slots)) {
        s = autotune_grids(S, nres);
        if (s == RT_OK && S->graph) {   // the graph holds the old grids
          cudaGraphExecDestroy(S->graph);
          S->graph = nullptr;
        }
      }
    }
    if (s == RT_OK && S->opts.graphs) s = capture_cycle(S);
    if (s != RT_OK) {
      fail(s);
      break;
    }
    // one restart cycle for every resident instance
    cudaError_t e = cudaSuccess;
    if (S->opts.graphs) {
      RT_NVTX("server restart cycle (graph)");
      e = cudaGraphLaunch(S->graph, S->st);
      if (e == cudaSuccess) count_launches(S->graph_kernels);
    } else {
      RT_NVTX("server restart cycle (direct launches)");
      s = enqueue_batch_cycle(S, S->st);
      if (s != RT_OK) {
        fail(s);
        break;
      }
      e = cudaGetLastError();
    }
    S->cycles.fetch_add(1);
    hs.resize(S->slots.size());
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(hs.data(), S->d_status, hs.size() * sizeof(InstStatus), cudaMemcpyDeviceToHost, S->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->st);
    if (e != cudaSuccess) {
      set_error("batch cycle failed: %s", cudaGetErrorString(e));
      fail(RT_ECUDA);
      break;
    }
    // retire finished instances
    int nres = 0;
    for (size_t q = 0; q < S->slots.size(); ++q) {
      Instance* in = S->slots[q];
      if (!in) continue;
      in->cycles += 1;
      const InstStatus& st = hs[q];
      rt_status fin = RT_EPENDING;
      if (st.rel != st.rel) fin = RT_ENUMERIC;
      else if (st.rel < in->req->rtol) fin = RT_OK;
      else if (st.iters >= in->req->maxit) fin = RT_ENOTCONV;
      else if (st.breakdown && st.kdone == 0) fin = RT_EBREAKDOWN;
      else if (st.kstop == 0) fin = RT_ENOTCONV;
      else if (in->req->cancel.load() || (in->req->deadline > 0.0 && wall_ms() > in->req->deadline))
        fin = RT_ECANCELED;
      if (fin != RT_EPENDING) {
        finish_request(S, in, st, fin);
        free_instance(S, in);
        delete in;
        S->slots[q] = nullptr;
      } else {
        ++nres;
      }
    }
    S->resident.store(nres);
  }
  for (Instance*& in : S->slots)
    if (in) {
      free_instance(S, in);
      delete in;
      in = nullptr;
    }
}

}  // namespace

}  // namespace rt

using namespace rt;

struct rt_server {
  rt::Server S;
};

extern "C" {

void rt_server_opts_default(rt_server_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof *o);
  o->mem_budget_bytes = (int64_t)8 << 30;
  o->max_slots = 64;
  o->restart = 30;
  o->precond = RT_PREC_LOCAL_LAMBDA;
  o->precision = RT_PRECISION_FP64;
  o->autotune = 1;
  o->graphs = 1;
}

static rt_status create_server(const rt_server_opts* opts, const rt_allocator* hook, rt_server** out) {
  RT_NVTX("rt_server_create");
  clear_error();
  if (!opts || !out) { set_error("opts and out are required"); return RT_EINVAL; }
  *out = nullptr;
  if (opts->max_slots < 1 || opts->max_slots > 4096) { set_error("max_slots must be in [1,4096]"); return RT_EINVAL; }
  if (opts->restart < 1 || opts->restart > kMaxRestart) { set_error("restart must be in [1,%d]", kMaxRestart); return RT_EINVAL; }
  if (opts->precond < RT_PREC_NONE || opts->precond > RT_PREC_LOCAL_LAMBDA) { set_error("bad precond"); return RT_EINVAL; }
  if (opts->precision != RT_PRECISION_FP64 && opts->precision != RT_PRECISION_FP32_REFINE) { set_error("bad precision"); return RT_EINVAL; }
  if (opts->mem_budget_bytes < ((int64_t)1 << 20)) { set_error("mem_budget_bytes must be >= 1 MiB"); return RT_EINVAL; }
  if (hook && (!hook->alloc || !hook->release)) { set_error("the allocator needs both alloc and release"); return RT_EINVAL; }
  rt_server* srv = new (std::nothrow) rt_server();
  if (!srv) { set_error("host allocation failed"); return RT_ENOMEM; }
  Server* S = &srv->S;
  S->opts = *opts;
  cudaError_t e = cudaGetDevice(&S->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&S->sms, cudaDevAttrMultiProcessorCount, S->device);
  if (e != cudaSuccess) {
    set_error("no CUDA device: %s", cudaGetErrorString(e));
    delete srv;
    return RT_ECUDA;
  }
  e = cudaStreamCreateWithFlags(&S->st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    set_error("server stream creation failed: %s", cudaGetErrorString(e));
    rt_server_destroy(srv);
    return RT_ECUDA;
  }
  if (hook) {
    S->hook = make_hook_allocator(hook, S->st);
    if (!S->hook) {
      set_error("host allocation failed");
      rt_server_destroy(srv);
      return RT_ENOMEM;
    }
  }
  rt_status s = S->arena.init((size_t)opts->mem_budget_bytes, S->hook);
  if (s != RT_OK) {
    rt_server_destroy(srv);
    return s;
  }
  S->slots.assign(opts->max_slots, nullptr);
  S->grid_h = 4 * S->sms;
  S->grid_g = 8 * S->sms;
  S->grid_v = 4 * S->sms;
  S->grid_i = (opts->max_slots + kInstThreads - 1) / kInstThreads;
  e = srv_alloc(S, (void**)&S->d_insts, sizeof(InstDev) * opts->max_slots);
  if (e == cudaSuccess) e = srv_alloc(S, (void**)&S->d_status, sizeof(InstStatus) * opts->max_slots);
  if (e == cudaSuccess) e = srv_alloc(S, (void**)&S->d_counts, sizeof(Counts));
  if (e == cudaSuccess) e = srv_alloc(S, (void**)&S->d_new_counts, sizeof(Counts));
  if (e == cudaSuccess) e = srv_alloc(S, (void**)&S->d_wl_i, sizeof(int) * opts->max_slots);
  if (e == cudaSuccess) e = srv_alloc(S, (void**)&S->d_wl_new_i, sizeof(int) * opts->max_slots);
  if (e != cudaSuccess) {
    set_error("server setup failed: %s", cudaGetErrorString(e));
    rt_server_destroy(srv);
    return e == cudaErrorMemoryAllocation ? RT_ENOMEM : RT_ECUDA;
  }
  S->worker = std::thread(worker_main, S);
  *out = srv;
  return RT_OK;
}

rt_status rt_server_create(const rt_server_opts* opts, rt_server** out) { return create_server(opts, nullptr, out); }

rt_status rt_server_create_with_allocator(const rt_server_opts* opts, const rt_allocator* allocator,
                                          rt_server** out) {
  return create_server(opts, allocator, out);
}

rt_status rt_batch_submit(rt_server* srv, const rt_problem_desc* desc, const rt_solver_opts* opts, uint64_t* ticket) {
  clear_error();
  if (!srv || !desc || !ticket) { set_error("srv, desc and ticket are required"); return RT_EINVAL; }
  RT_TRY(validate_desc(desc));
  if (desc->Ns > 4096) { set_error("batched instances need Ns <= 4096"); return RT_EINVAL; }
  if (desc->form != RT_FORM_I) { set_error("the batch server solves I-form problems only"); return RT_EINVAL; }
  if (desc->formal_solver == RT_FS_DELO_PARABOLIC) {
    set_error("the batch server does not take the DELO-parabolic formal solver");
    return RT_EINVAL;
  }
  Server* S = &srv->S;
  auto rq = std::make_unique<Request>();
  rq->desc = *desc;
  rq->tau.assign(desc->tau, desc->tau + desc->Ns);
  rq->desc.tau = rq->tau.data();
  if (desc->B) {
    rq->B.assign(desc->B, desc->B + desc->Ns);
    rq->desc.B = rq->B.data();
  }
  if (desc->phi) {
    rq->phi.assign(desc->phi, desc->phi + desc->Nnu);
    rq->desc.phi = rq->phi.data();
  }
  if (opts) {
    if (!(opts->rtol > 0.0) || opts->maxit < 1) { set_error("rtol must be > 0 and maxit >= 1"); return RT_EINVAL; }
    rq->rtol = opts->rtol;
    rq->maxit = opts->maxit;
    if (opts->deadline_ms < 0.0 || opts->deadline_ms != opts->deadline_ms) {
      set_error("deadline_ms must be >= 0");
      return RT_EINVAL;
    }
  }
  rq->t_submit = wall_ms();
  if (opts && opts->deadline_ms > 0.0) rq->deadline = rq->t_submit + opts->deadline_ms;
  rq->info.status = RT_EPENDING;
  const uint64_t t = S->next_ticket.fetch_add(1);
  rq->ticket = t;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->worker_status != RT_OK) {
      set_error("server failed: %s", S->worker_error.c_str());
      return S->worker_status;
    }
    S->pending.push_back(rq.get());
    S->requests[t] = std::move(rq);
  }
  S->cv.notify_one();
  *ticket = t;
  return RT_OK;
}

rt_status rt_poll(rt_server* srv, uint64_t ticket, rt_solve_info* info, double* x_host) {
  clear_error();
  if (!srv) { set_error("srv is NULL"); return RT_EINVAL; }
  Server* S = &srv->S;
  std::unique_ptr<Request> done;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->requests.find(ticket);
    if (it == S->requests.end()) { set_error("unknown ticket %llu", (unsigned long long)ticket); return RT_EINVAL; }
    if (!it->second->done) {
      if (info) {
        memset(info, 0, sizeof *info);
        info->status = RT_EPENDING;
      }
      return RT_EPENDING;
    }
    done = std::move(it->second);
    S->requests.erase(it);
  }
  if (info) *info = done->info;
  if (x_host) {
    if (!done->x.empty()) memcpy(x_host, done->x.data(), done->x.size() * sizeof(double));
    else   // never admitted (cancelled while queued, or no room in the budget): zeros
      memset(x_host, 0, (size_t)2 * done->desc.Ns * done->desc.Nmu * done->desc.Nnu * sizeof(double));
  }
  return done->info.status;
}

rt_status rt_batch_cancel(rt_server* srv, uint64_t ticket) {
  clear_error();
  if (!srv) { set_error("srv is NULL"); return RT_EINVAL; }
  Server* S = &srv->S;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->requests.find(ticket);
  if (it == S->requests.end()) { set_error("unknown ticket %llu", (unsigned long long)ticket); return RT_EINVAL; }
  Request* rq = it->second.get();
  if (rq->done) return RT_OK;
  for (auto q = S->pending.begin(); q != S->pending.end(); ++q)
    if (*q == rq) {   // still queued: it ends now
      S->pending.erase(q);
      rq->info.status = RT_ECANCELED;
      rq->t_done = wall_ms();
      rq->info.t_total_ms = rq->t_done - rq->t_submit;
      rq->done = true;
      S->completed.fetch_add(1);
      return RT_OK;
    }
  rq->cancel.store(true);   // admitted: the worker ends it after the current cycle
  return RT_OK;
}

rt_status rt_server_stats_get(rt_server* srv, rt_server_stats* out) {
  clear_error();
  if (!srv || !out) { set_error("srv and out are required"); return RT_EINVAL; }
  Server* S = &srv->S;
  memset(out, 0, sizeof *out);
  {
    std::lock_guard<std::mutex> lk(S->mu);
    out->queued = (int32_t)S->pending.size();
  }
  out->resident = S->resident.load();
  out->arena_in_use = (int64_t)S->arena.in_use();
  out->arena_largest_free = (int64_t)S->arena.largest_hole();
  out->cycles = S->cycles.load();
  out->completed = S->completed.load();
  out->grid_quad = S->grid_h;
  out->grid_formal = S->grid_g;
  out->grid_vec = S->grid_v;
  out->tuned = S->tuned ? 1 : 0;
  return RT_OK;
}

rt_status rt_server_destroy(rt_server* srv) {
  if (!srv) return RT_OK;
  Server* S = &srv->S;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  if (S->worker.joinable()) S->worker.join();
  drop_graph(S);
  // a caller's allocator may hand a released block to its next user at once
  if (S->hook) cudaDeviceSynchronize();
  void* ptrs[] = {S->d_insts, S->d_status, S->d_counts, S->d_new_counts, S->d_wl_i, S->d_wl_new_i, S->d_wl_h,
                  S->d_wl_c, S->d_wl_g64, S->d_wl_g32, S->d_wl_new_c};
  for (void* p : ptrs) srv_free(S, p);
  S->arena.teardown();
  if (S->st) cudaStreamDestroy(S->st);
  if (S->cap) cudaStreamDestroy(S->cap);
  delete S->hook;
  S->hook = nullptr;
  delete srv;
  return RT_OK;
}

}  // extern "C"

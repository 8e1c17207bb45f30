// Krylov solvers on the device (Sect. 2 of the paper): restarted GMRES(m)
// with modified Gram-Schmidt Arnoldi (in block form) and Givens rotations,
// BiCGSTAB, CGS and preconditioned Richardson, plus FP32-operator iterative
// refinement.
//
// Design:
//  * every reduction is deterministic: a fixed grid writes one partial per
//    block, and the consumer sums the partials in a fixed order (each block
//    of the consumer kernel redundantly, so no extra launch is needed);
//  * all scalars (Hessenberg matrix, rotations, alpha/omega/rho) stay in
//    device memory and are updated by one thread -- of a scalar kernel, or
//    of a dedicated CTA of the kernel that needs them next (the Givens
//    rotations run in a CTA of the scaling kernel, or of the next step's
//    quadrature kernel) -- so a whole GMRES restart cycle (m Arnoldi steps,
//    the least-squares solve, the update of x and the true residual) is one
//    CUDA graph launch followed by one host read of the convergence state;
//  * a step index baked into each kernel of the cycle graph is compared with
//    the device counter `kstop`: once the residual estimate passes the
//    tolerance the remaining kernels of the cycle return at once.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <chrono>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>

#include <cuda.h>

#include "rt_common.cuh"

namespace rt {

namespace {

constexpr int kVecThreads = kBlockVec;
constexpr int kWorkVecs = 9;

template <typename T>
__device__ __forceinline__ T wsum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block sum in a fixed order; result valid in thread 0
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = wsum(v);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  __syncthreads();
  return s;
}

// sum of G partials in a fixed order (lane-strided, then a fixed shuffle tree);
// every thread of the calling warp gets the result
__device__ __forceinline__ double sum_partials_warp(const double* __restrict__ part, int G) {
  return partials_sum_warp(part, G);
}

// broadcast of sum_partials to the whole block
__device__ __forceinline__ double block_partials(const double* __restrict__ part, int G) {
  __shared__ double bc;
  if (threadIdx.x < 32) {
    const double s = sum_partials_warp(part, G);
    if (threadIdx.x == 0) bc = s;
  }
  __syncthreads();
  const double v = bc;
  __syncthreads();
  return v;
}

// sqrt(sum of the partials) and its inverse (0 for a zero norm), computed
// once per block by thread 0 (FP64 square roots and divisions are long
// sequences on this GPU's narrow FP64 pipe) and broadcast to the block
__device__ __forceinline__ double block_norm_inv(const double* __restrict__ part, int G, double* hn_out) {
  __shared__ double nb[2];
  if (threadIdx.x < 32) {
    const double s = sum_partials_warp(part, G);
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

// ------------------------------------------------------------------ kernels
// Grid-stride loops unrolled by kU with all loads of a round issued before
// any arithmetic, so each thread keeps kU independent loads in flight.
constexpr int kU = 4;

// skip test shared by the kernels of a captured iteration: GMRES kernels of
// Arnoldi step `step` skip once step >= *kstop; BiCGSTAB/CGS kernels skip
// once *done is set
__device__ __forceinline__ bool gated(const int* kstop, int step, const int* done) {
  return (kstop && step >= *kstop) || (done && *done);
}

__global__ void __launch_bounds__(kVecThreads) k_dot(const double* __restrict__ a, const double* __restrict__ b,
                                                     int64_t N, double* __restrict__ part, const int* kstop, int step,
                                                     const int* done) {
  if (gated(kstop, step, done)) return;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double s = 0.0;
  for (; i + (kU - 1) * stride < N; i += kU * stride) {
    double av[kU], bv[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) { av[u] = a[i + u * stride]; bv[u] = b[i + u * stride]; }
#pragma unroll
    for (int u = 0; u < kU; ++u) s = fma(av[u], bv[u], s);
  }
  for (; i < N; i += stride) s = fma(a[i], b[i], s);
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// two dot products at once: part[0..G) = <a,b>, part[G..2G) = <c,d>
__global__ void __launch_bounds__(kVecThreads) k_dot2(const double* __restrict__ a, const double* __restrict__ b,
                                                      const double* __restrict__ c, const double* __restrict__ d,
                                                      int64_t N, double* __restrict__ part, const int* done) {
  if (done && *done) return;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double s = 0.0, t = 0.0;
  for (; i + (kU - 1) * stride < N; i += kU * stride) {
    double av[kU], bv[kU], cv[kU], dv[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      av[u] = a[i + u * stride];
      bv[u] = b[i + u * stride];
      cv[u] = c[i + u * stride];
      dv[u] = d[i + u * stride];
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      s = fma(av[u], bv[u], s);
      t = fma(cv[u], dv[u], t);
    }
  }
  for (; i < N; i += stride) {
    s = fma(a[i], b[i], s);
    t = fma(c[i], d[i], t);
  }
  s = block_sum(s);
  t = block_sum(t);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s;
    part[gridDim.x + blockIdx.x] = t;
  }
}

// MGS pass: h = sum(part_in); w -= h * vprev; partial <w, vnext> (or <w,w>).
// The first round's loads do not depend on h, so they are issued before the
// block sums the previous pass's partials and their latency overlaps it.
__global__ void __launch_bounds__(kVecThreads) k_mgs(double* __restrict__ w, const double* __restrict__ vprev,
                                                     const double* __restrict__ vnext, int64_t N,
                                                     const double* __restrict__ part_in, double* __restrict__ part_out,
                                                     double* __restrict__ hslot, const int* kstop, int step) {
  if (kstop && step >= *kstop) return;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const double* __restrict__ vn = vnext ? vnext : w;
  double wv[kU], pv[kU], nv[kU];
  const bool first = i + (kU - 1) * stride < N;
  if (first) {
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      wv[u] = w[i + u * stride];
      pv[u] = vprev[i + u * stride];
      if (vnext) nv[u] = vnext[i + u * stride];
    }
  }
  const double h = block_partials(part_in, gridDim.x);
  if (blockIdx.x == 0 && threadIdx.x == 0) *hslot = h;
  double s = 0.0;
  for (bool loaded = first; i + (kU - 1) * stride < N; i += kU * stride, loaded = false) {
    if (!loaded) {
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        wv[u] = w[i + u * stride];
        pv[u] = vprev[i + u * stride];
        if (vnext) nv[u] = vnext[i + u * stride];
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const double wi = fma(-h, pv[u], wv[u]);
      w[i + u * stride] = wi;
      s = fma(wi, vnext ? nv[u] : wi, s);
    }
  }
  for (; i < N; i += stride) {
    const double wi = fma(-h, vprev[i], w[i]);
    w[i] = wi;
    s = fma(wi, vnext ? vn[i] : wi, s);
  }
  s = block_sum(s);
  if (threadIdx.x == 0) part_out[blockIdx.x] = s;
}

// v = w / ||w|| with ||w|| from the partials, written to *hout
__global__ void __launch_bounds__(kVecThreads) k_norm_out(const double* __restrict__ w, double* __restrict__ v,
                                                          int64_t N, const double* __restrict__ part_in,
                                                          double* __restrict__ hout) {
  double hn;
  const double inv = block_norm_inv(part_in, gridDim.x, &hn);
  if (blockIdx.x == 0 && threadIdx.x == 0) *hout = hn;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = w[i] * inv;
}

// ------------------------------------------------- block MGS Arnoldi step
// The GMRES Arnoldi step orthogonalises w against v_0..v_j in passes of
// kGramB basis vectors.  With r_k = <w, v_k> taken before a block's updates,
// modified Gram-Schmidt's coefficients satisfy exactly
//     h_k = <w - sum_{l<k} h_l v_l, v_k> = r_k - sum_{l<k} h_l <v_l, v_k>
// (l, k in the block), so each pass sums the previous pass's dots, solves
// this small triangular system with the stored Gram entries <v_l, v_k>,
// applies all of the block's updates to w element by element (in MGS order)
// and accumulates the dots of the updated w with the next block.  One launch
// per block instead of one per basis vector; the same FP64 operations per
// element as MGS.  The last pass also accumulates ||w||^2 and the dots of
// the final w with the vectors of its block: those are the Gram entries of
// v_{j+1} that the next step reads (v_{j+1} shares a block only with them).
// The normalisation v_{j+1} = w / ||w|| is then a plain scaling pass, whose
// last CTA folds h_{j+1,j} and the Gram row and rotates the Hessenberg
// column.
//
// The FP64 pipe bounds these kernels, so the reductions are kept short: one
// CTA per resident slot (a single wave, several elements per thread) and a
// transposing warp reduction of the four accumulators (6 FP64 additions per
// thread instead of 20).
constexpr int kB = kGramB;
// shape of the block-pass kernels: one wave of kMgsCtasPerSm CTAs of
// kMgsThreads per SM (64 registers a thread)
constexpr int kMgsThreads = 512, kMgsCtasPerSm = 2;

// block sums of s[0..kB-1] in a fixed order; sum k < n goes to
// out[k * gridDim.x + blockIdx.x].  Launch with kMgsThreads threads.
__device__ __forceinline__ void block_sum4_out(const double* s, int n, double* __restrict__ out) {
  constexpr int NW = kMgsThreads / 32;
  static_assert(kB == 4 && kB * NW <= 128 && (NW & (NW - 1)) == 0, "reduction layout");
  __shared__ double red[kB][NW];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const double t = warp_sum4(s);
  if ((lane & 7) == 0) red[lane >> 3][warp] = t;
  __syncthreads();
  if (threadIdx.x < kB * NW) {   // warps 0 and 1: value k = tid / NW, source warp tid % NW
    const int k = threadIdx.x / NW, src = threadIdx.x % NW;
    double x = red[k][src];
#pragma unroll
    for (int o = NW / 2; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (src == 0 && k < n) out[(size_t)k * gridDim.x + blockIdx.x] = x;
  }
}

// warps 0..n-1 each sum one set of G partials (fixed order) into out[k]
__device__ __forceinline__ void sum_sets(const double* __restrict__ part, int G, int n, double* out) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp < n) {
    const double s = sum_partials_warp(part + (size_t)warp * G, G);
    if (lane == 0) out[warp] = s;
  }
  __syncthreads();
}

// The three kernels are launched as programmatic dependents of the kernel
// before them (launch_pdl): a CTA may start while the previous grid drains,
// runs what does not depend on it (the gate, the basis-vector loads of its
// first element, the Gram entries), then waits in griddepcontrol.wait until
// that grid has finished and its writes are visible.  The gate counter is
// read before that wait.  It is written only by the Givens update of the step
// before (the scaling kernel, or the first CTA of this step's quadrature
// kernel), which finished before the kernels of this step's apply passed
// their own waits.  The counter only falls within a cycle (at convergence),
// so a read that still saw its earlier value would run a block pass of a
// step past convergence: work on the discarded part of the basis and of the
// Hessenberg matrix, which nothing of the cycle reads afterwards.

// Each pass sweeps the vectors in the opposite direction to the pass before
// (rev): it starts on the elements the previous pass touched last, which are
// still in L2 -- w and the vectors whose dots that pass just formed.

// The block sizes are template parameters: a DFMA under a false predicate
// still takes its slot on the FP64 pipe, so a runtime guard "k < nb" would
// cost every pass the work of a full block.  Passes before the last always
// have kB vectors.

// first kernel of Arnoldi step j: partial dots <w, v_k>, k < NK
template <int NK>
__global__ void __launch_bounds__(kMgsThreads, kMgsCtasPerSm) k_bdot(const double* __restrict__ w, const double* __restrict__ V,
                                                        int64_t N, double* __restrict__ part_out, int j, int rev,
                                                        const int* kstop) {
  constexpr int nk = NK;
  if (kstop && j >= *kstop) return;
  pdl_launch_dependents();
  pdl_wait();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  double s[kB] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += stride) {
    const int64_t e = rev ? N - 1 - i : i;
    const double wi = w[e];
    double vv[kB];
#pragma unroll
    for (int k = 0; k < kB; ++k)
      if (k < nk) vv[k] = V[(size_t)k * N + e];
#pragma unroll
    for (int k = 0; k < kB; ++k)
      if (k < nk) s[k] = fma(wi, vv[k], s[k]);
  }
  block_sum4_out(s, nk, part_out);
}

// one block pass of Arnoldi step j over v_{i0} .. v_{i0+NB-1}; with NN > 0
// the dots of the updated w with the next NN vectors, with NN == 0 (the last
// block) ||w||^2 and the Gram dots <w, v_{i0+k}>, k < ng (= NB when v_{j+1}
// shares the block, else 0)
template <int NB, int NN>
__global__ void __launch_bounds__(kMgsThreads, kMgsCtasPerSm) k_bmgs(double* __restrict__ w, const double* __restrict__ V,
                                                        int64_t N, int i0, const double* __restrict__ part_in,
                                                        double* __restrict__ part_out, double* __restrict__ hcol,
                                                        const double* __restrict__ gram, int j, int rev,
                                                        const int* kstop) {
  static_assert(NB >= 1 && NB <= kB && NN >= 0 && NN <= kB && (NN == 0 || NB == kB), "block shape");
  constexpr int nb = NB, nn = NN, ng = NN == 0 && NB < kB ? NB : 0;
  if (kstop && j >= *kstop) return;
  pdl_launch_dependents();
  const int G = gridDim.x;
  const double* __restrict__ vb = V + (size_t)i0 * N;
  const double* __restrict__ vn = V + (size_t)(i0 + nb) * N;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  // the first element's basis-vector loads depend neither on h nor on the
  // previous pass: issue them first
  double wv = 0.0, bv[kB], nv[kB];
  auto load_v = [&](int64_t e) {
#pragma unroll
    for (int k = 0; k < kB; ++k) {
      if (k < nb) bv[k] = vb[(size_t)k * N + e];
      if (k < nn) nv[k] = vn[(size_t)k * N + e];
    }
  };
  if (i < N) load_v(rev ? N - 1 - i : i);
  // the block's Gram entries <v_{i0+l}, v_{i0+k}> (l < k), fetched by the
  // warp after the partial sums while those are being summed
  __shared__ double rs[kB], hs[kB], gs[kB][kB];
  const int t = threadIdx.x - 32 * kB;
  if (t >= 0 && t < kB * kB) {
    const int k = t / kB, d = t % kB;
    gs[k][d] = k < nb && d >= 1 && d <= k ? gram[(i0 + k) * kB + d] : 0.0;
  }
  pdl_wait();
  if (i < N) wv = w[rev ? N - 1 - i : i];
  sum_sets(part_in, G, nb, rs);
  if (threadIdx.x == 0) {
    for (int k = 0; k < nb; ++k) {
      double h = rs[k];
      for (int l = 0; l < k; ++l) h -= hs[l] * gs[k][k - l];
      hs[k] = h;
      if (blockIdx.x == 0) hcol[i0 + k] = h;
    }
  }
  __syncthreads();
  double h[kB];
#pragma unroll
  for (int k = 0; k < kB; ++k) h[k] = k < nb ? hs[k] : 0.0;
  double s[kB] = {0.0, 0.0, 0.0, 0.0};
  for (; i < N; i += stride) {
    const int64_t e = rev ? N - 1 - i : i;
    // software pipeline: the next element's loads are issued before this
    // element's FP64 work
    const int64_t i2 = i + stride;
    double wv2 = 0.0, bv2[kB], nv2[kB];
    if (i2 < N) {
      const int64_t e2 = rev ? N - 1 - i2 : i2;
      wv2 = w[e2];
#pragma unroll
      for (int k = 0; k < kB; ++k) {
        if (k < nb) bv2[k] = vb[(size_t)k * N + e2];
        if (k < nn) nv2[k] = vn[(size_t)k * N + e2];
      }
    }
    double wi = wv;
#pragma unroll
    for (int k = 0; k < kB; ++k)
      if (k < nb) wi = fma(-h[k], bv[k], wi);
    w[e] = wi;
    if constexpr (nn > 0) {
#pragma unroll
      for (int k = 0; k < kB; ++k)
        if (k < nn) s[k] = fma(wi, nv[k], s[k]);
    } else {
      s[0] = fma(wi, wi, s[0]);
#pragma unroll
      for (int k = 0; k < kB - 1; ++k)
        if (k < ng) s[1 + k] = fma(wi, bv[k], s[1 + k]);
    }
    wv = wv2;
#pragma unroll
    for (int k = 0; k < kB; ++k) {
      if (k < nb) bv[k] = bv2[k];
      if (k < nn) nv[k] = nv2[k];
    }
  }
  block_sum4_out(s, nn ? nn : 1 + ng, part_out);
}

// v_{j+1} = w / ||w|| by blocks 1..gridDim.x-1 (||w||^2 is set 0 of the last
// pass's partials, over Gp blocks).  Block 0, scheduled first, writes
// h_{j+1} = ||w|| to hcol[j+1] and the Gram row j+1: <v_{j+1}, v_{j+1-d}> =
// <w, v_{i0+k}> / ||w|| (set 1+k, d = ng - k, k < ng), then, inside GMRES
// (gm set), applies the Givens rotations to column j.  Three CTAs fit on an
// SM, so the grid (one CTA per block-pass slot, plus block 0) is one wave;
// each thread loads its first elements while the norm is being formed.
constexpr int kScaleU = 4;
__global__ void __launch_bounds__(kVecThreads, 3) k_bscale(const double* __restrict__ w, double* __restrict__ V,
                                                           int64_t N, const double* __restrict__ part_in, int Gp,
                                                           int ng, double* __restrict__ hcol, double* __restrict__ gram,
                                                           GmresDev* gm, int m, int j, double* hist, int hist_cap,
                                                           int rev, const int* kstop) {
  if (kstop && j >= *kstop) return;
  pdl_wait();
  if (blockIdx.x == 0) {
    arnoldi_fold(part_in, Gp, ng, hcol, gram, gm, m, j, hist, hist_cap);
    return;
  }
  double* __restrict__ vo = V + (size_t)(j + 1) * N;
  const int64_t stride = (int64_t)(gridDim.x - 1) * blockDim.x;
  const int64_t i0 = (blockIdx.x - 1) * (int64_t)blockDim.x + threadIdx.x;
  double wv[kScaleU];
#pragma unroll
  for (int u = 0; u < kScaleU; ++u) {
    const int64_t i = i0 + u * stride;
    wv[u] = i < N ? w[rev ? N - 1 - i : i] : 0.0;
  }
  double hn;
  const double inv = block_norm_inv(part_in, Gp, &hn);
#pragma unroll
  for (int u = 0; u < kScaleU; ++u) {
    const int64_t i = i0 + u * stride;
    if (i < N) vo[rev ? N - 1 - i : i] = wv[u] * inv;
  }
  for (int64_t i = i0 + kScaleU * stride; i < N; i += stride) {
    const int64_t e = rev ? N - 1 - i : i;
    vo[e] = w[e] * inv;
  }
}

// the end of the last Arnoldi step of a cycle whose normalisations are done
// by the next step's apply (NormIn): the fold and the Givens rotations only
__global__ void k_arnoldi_tail(const double* __restrict__ part, int Gp, int ng, double* __restrict__ hcol,
                               double* __restrict__ gram, GmresDev* gm, int m, int j, double* hist, int hist_cap,
                               const int* kstop) {
  if (kstop && j >= *kstop) return;
  arnoldi_fold(part, Gp, ng, hcol, gram, gm, m, j, hist, hist_cap);
}

// the grid of the block-MGS passes: one CTA per resident slot
inline int mgs_grid(const Problem* P) {
  int64_t g = (P->Nop + kMgsThreads - 1) / kMgsThreads;
  const int cap = std::min(kMgsCtasPerSm * P->num_sms, kMaxPartials);
  return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

// back substitution H(0:k,0:k) y = g(0:k) in the textbook order: row k-1
// first, each row's sum running from g_i over l = i+1.. in increasing order,
// then one division.  The warp stages the triangle in shared memory (packed
// by columns; 103 KB for the longest cycle, 160 steps) and thread 0 runs the
// recurrence from there.  The order matters in FP32 refinement: a warp-tree
// sum of the same products changed the inner solves' iteration counts by up
// to 10%.  Dynamic shared memory for cycles of up to m steps: the packed
// triangle, then y.
inline size_t lsq_smem(int m) { return ((size_t)m * (m + 1) / 2 + (size_t)m) * sizeof(double); }

__global__ void k_lsq(GmresDev* gm, int m) {
  const int k = gm->kdone, lane = threadIdx.x;
  extern __shared__ double lsq_sm[];
  double* Hs = lsq_sm;                          // column l (rows 0..l) at l (l + 1) / 2
  double* ys = lsq_sm + (size_t)m * (m + 1) / 2;
  // the packed triangle, q = l (l + 1) / 2 + i, in rounds of 8 loads a lane
  // issued before any store (a column-by-column copy waited for each load)
  const int total = k * (k + 1) / 2;
  constexpr int U = 8;
  for (int q0 = 0; q0 < total; q0 += 32 * U) {
    double v[U];
    int dst[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int q = q0 + u * 32 + lane;
      dst[u] = q < total ? q : -1;
      if (q < total) {
        int l = (int)((sqrtf(8.0f * (float)q + 1.0f) - 1.0f) * 0.5f);
        while (l * (l + 1) / 2 > q) --l;           // exact column of q despite the rounding of sqrtf
        while ((l + 1) * (l + 2) / 2 <= q) ++l;
        v[u] = gm->H[l * (m + 1) + (q - l * (l + 1) / 2)];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (dst[u] >= 0) Hs[dst[u]] = v[u];
  }
  __syncwarp();
  if (lane == 0) {
    for (int i = k - 1; i >= 0; --i) {
      double s = gm->g[i];
      for (int l = i + 1; l < k; ++l) s -= Hs[l * (l + 1) / 2 + i] * ys[l];
      ys[i] = s / Hs[i * (i + 1) / 2 + i];
    }
  }
  __syncwarp();
  for (int i = lane; i < k; i += 32) gm->y[i] = ys[i];
}

// t = sum_{i<k} y_i V_i; mode 0: x += t, 1: x += dinv*t, 2: t stored for P^{-1}
// (with no step done, t = 0, so that the x += P^{-1} t that follows adds nothing
// rather than the previous cycle's update once more)
__global__ void __launch_bounds__(kVecThreads) k_combine(const double* __restrict__ V, int64_t N,
                                                         const GmresDev* gm, double* __restrict__ x,
                                                         const double* __restrict__ dinv, double* __restrict__ t,
                                                         int mode) {
  const int k = gm->kdone;
  __shared__ double ys[kMaxRestart];
  for (int i = threadIdx.x; i < k; i += blockDim.x) ys[i] = gm->y[i];
  __syncthreads();
  if (k == 0) {
    if (mode == 2)
      for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x)
        t[n] = 0.0;
    return;
  }
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < k; ++i) s = fma(ys[i], V[(int64_t)i * N + n], s);
    if (mode == 0) x[n] += s;
    else if (mode == 1) x[n] = fma(dinv[n], s, x[n]);
    else t[n] = s;
  }
}

// x += z
__global__ void __launch_bounds__(kVecThreads) k_axpy1(double* __restrict__ x, const double* __restrict__ z, int64_t N) {
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x)
    x[n] += z[n];
}

// r = b - Ax; partial ||r||^2
__global__ void __launch_bounds__(kVecThreads) k_residual(const double* __restrict__ b, const double* __restrict__ Ax,
                                                          double* __restrict__ r, int64_t N, double* __restrict__ part) {
  double s = 0.0;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
    const double v = b[n] - Ax[n];
    r[n] = v;
    s = fma(v, v, s);
  }
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// start of a cycle: beta = ||r||, v_0 = r / beta, g = beta e_1
__global__ void __launch_bounds__(kVecThreads) k_cycle_start(const double* __restrict__ r, double* __restrict__ v0,
                                                             int64_t N, const double* __restrict__ part, GmresDev* gm,
                                                             int m) {
  double rn;
  const double inv = block_norm_inv(part, gridDim.x, &rn);
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x)
    v0[n] = r[n] * inv;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    gm->rnorm = rn;
    gm->rel = rn / gm->bnorm;
    for (int i = 0; i <= m; ++i) gm->g[i] = 0.0;
    gm->g[0] = rn;
    gm->kdone = 0;
    int left = gm->maxit - gm->iters;
    gm->kstop = left < m ? (left > 0 ? left : 0) : m;
    if (!(gm->rel >= gm->tol)) gm->kstop = 0;  // converged (or NaN): no steps
  }
}

__global__ void k_set_bnorm(const double* __restrict__ part, int G, GmresDev* gm) {
  if (threadIdx.x < 32) {
    const double s = sum_partials_warp(part, G);
    if (threadIdx.x == 0) gm->bnorm = sqrt(s);
  }
}

// ---------------------------------------------------- BiCGSTAB / CGS kernels
__device__ __forceinline__ double fin(const double* part, int G) {  // single-warp use
  return sum_partials_warp(part, G);
}

// scalar kernels run with one warp
__global__ void k_bc_init(BicgDev* bc, const double* part, int G) {
  // part: [<r,r> | <rhat,r>]
  const double rr = fin(part, G), rho = fin(part + G, G);
  if (threadIdx.x == 0) {
    bc->rel = sqrt(rr) / bc->bnorm;
    bc->rho = rho;
    bc->rho_old = 1.0;
    bc->alpha = 1.0;
    bc->omega = 1.0;
    bc->beta = 0.0;
    bc->done = !(bc->rel >= bc->tol) ? 1 : 0;
    if (bc->rel != bc->rel) bc->done = 3;
    if (!bc->done && rho == 0.0) bc->done = 2;
  }
}

// alpha = rho / <rhat, v>
__global__ void k_bc_alpha(BicgDev* bc, const double* part, int G) {
  if (bc->done) return;
  const double rv = fin(part, G);
  if (threadIdx.x == 0) {
    if (rv == 0.0) { bc->done = 2; return; }
    bc->alpha = bc->rho / rv;
  }
}

// ---- BiCGSTAB
// p = r + beta (p - omega v)
__global__ void __launch_bounds__(kVecThreads) k_bs_p(double* __restrict__ p, const double* __restrict__ r,
                                                      const double* __restrict__ v, int64_t N, const BicgDev* bc) {
  if (bc->done) return;
  const double beta = bc->beta, omega = bc->omega;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x)
    p[n] = fma(beta, fma(-omega, v[n], p[n]), r[n]);
}

// s = r - alpha v, partial ||s||^2
__global__ void __launch_bounds__(kVecThreads) k_bs_s(double* __restrict__ s, const double* __restrict__ r,
                                                      const double* __restrict__ v, int64_t N, const BicgDev* bc,
                                                      double* __restrict__ part) {
  if (bc->done) return;
  const double alpha = bc->alpha;
  double acc = 0.0;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
    const double v2 = fma(-alpha, v[n], r[n]);
    s[n] = v2;
    acc = fma(v2, v2, acc);
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// half-step test on ||s||
__global__ void k_bs_check_s(BicgDev* bc, const double* part, int G) {
  if (bc->done) return;
  const double ss = fin(part, G);
  if (threadIdx.x == 0) {
    const double rel = sqrt(ss) / bc->bnorm;
    bc->iters += 1;
    if (!(rel >= bc->tol)) {
      bc->rel = rel;
      bc->half = 1;
      bc->done = (rel != rel) ? 3 : 1;
    }
  }
}

// omega = <t,s>/<t,t>
__global__ void k_bs_omega(BicgDev* bc, const double* part, int G) {
  if (bc->done) return;
  const double ts = fin(part, G), tt = fin(part + G, G);
  if (threadIdx.x == 0) {
    if (tt == 0.0) { bc->done = 2; return; }
    bc->omega = ts / tt;
  }
}

// acc += alpha p + omega s (the half-step: acc += alpha p); r = s - omega t;
// partials ||r||^2 and <rhat, r>
__global__ void __launch_bounds__(kVecThreads) k_bs_update(double* __restrict__ acc, const double* __restrict__ p,
                                                           const double* __restrict__ s, const double* __restrict__ t,
                                                           double* __restrict__ r, const double* __restrict__ rhat,
                                                           int64_t N, const BicgDev* bc, double* __restrict__ part) {
  if (bc->done == 1 && bc->half) {
    // converged on s: finish the direction update only (once)
    if (bc->half == 1) {
      const double alpha = bc->alpha;
      for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x)
        acc[n] = fma(alpha, p[n], acc[n]);
    }
    return;
  }
  if (bc->done) return;
  const double alpha = bc->alpha, omega = bc->omega;
  double a1 = 0.0, a2 = 0.0;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
    acc[n] = fma(alpha, p[n], fma(omega, s[n], acc[n]));
    const double rn = fma(-omega, t[n], s[n]);
    r[n] = rn;
    a1 = fma(rn, rn, a1);
    a2 = fma(rhat[n], rn, a2);
  }
  a1 = block_sum(a1);
  a2 = block_sum(a2);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = a1;
    part[gridDim.x + blockIdx.x] = a2;
  }
}

__global__ void k_bs_check_r(BicgDev* bc, const double* part, int G, double* hist, int hist_cap) {
  if (bc->done == 1 && bc->half == 1) {
    if (threadIdx.x == 0) {
      bc->half = 2;  // the direction update of the half step has been applied
      if (hist && bc->iters - 1 < hist_cap) hist[bc->iters - 1] = bc->rel;
    }
    return;
  }
  if (bc->done) return;
  const double rr = fin(part, G), rho = fin(part + G, G);
  if (threadIdx.x == 0) {
    bc->rel = sqrt(rr) / bc->bnorm;
    if (hist && bc->iters - 1 < hist_cap) hist[bc->iters - 1] = bc->rel;
    if (bc->rel != bc->rel) { bc->done = 3; return; }
    if (!(bc->rel >= bc->tol)) { bc->done = 1; return; }
    if (bc->omega == 0.0 || rho == 0.0) { bc->done = 2; return; }
    bc->beta = (rho / bc->rho) * (bc->alpha / bc->omega);
    bc->rho = rho;
    if (bc->iters >= bc->maxit) bc->done = 4;
  }
}

// ---- CGS
// u = r + beta q; p = u + beta (q + beta p)
__global__ void __launch_bounds__(kVecThreads) k_cgs_up(double* __restrict__ u, double* __restrict__ p,
                                                        const double* __restrict__ r, const double* __restrict__ q,
                                                        int64_t N, const BicgDev* bc) {
  if (bc->done) return;
  const double beta = bc->beta;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
    const double un = fma(beta, q[n], r[n]);
    u[n] = un;
    p[n] = fma(beta, fma(beta, p[n], q[n]), un);
  }
}

// q = u - alpha vhat; w = u + q; acc += alpha w
__global__ void __launch_bounds__(kVecThreads) k_cgs_q(double* __restrict__ q, double* __restrict__ w,
                                                       double* __restrict__ acc, const double* __restrict__ u,
                                                       const double* __restrict__ vh, int64_t N, const BicgDev* bc) {
  if (bc->done) return;
  const double alpha = bc->alpha;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
    const double qn = fma(-alpha, vh[n], u[n]);
    q[n] = qn;
    const double wn = u[n] + qn;
    w[n] = wn;
    acc[n] = fma(alpha, wn, acc[n]);
  }
}

// r -= alpha qhat; partials ||r||^2, <rhat, r>
__global__ void __launch_bounds__(kVecThreads) k_cgs_r(double* __restrict__ r, const double* __restrict__ qh,
                                                       const double* __restrict__ rhat, int64_t N, const BicgDev* bc,
                                                       double* __restrict__ part) {
  if (bc->done) return;
  const double alpha = bc->alpha;
  double a1 = 0.0, a2 = 0.0;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
    const double rn = fma(-alpha, qh[n], r[n]);
    r[n] = rn;
    a1 = fma(rn, rn, a1);
    a2 = fma(rhat[n], rn, a2);
  }
  a1 = block_sum(a1);
  a2 = block_sum(a2);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = a1;
    part[gridDim.x + blockIdx.x] = a2;
  }
}

__global__ void k_cgs_check(BicgDev* bc, const double* part, int G, double* hist, int hist_cap) {
  if (bc->done) return;
  const double rr = fin(part, G), rho = fin(part + G, G);
  if (threadIdx.x == 0) {
    bc->iters += 1;
    bc->rel = sqrt(rr) / bc->bnorm;
    if (hist && bc->iters - 1 < hist_cap) hist[bc->iters - 1] = bc->rel;
    if (bc->rel != bc->rel) { bc->done = 3; return; }
    if (!(bc->rel >= bc->tol)) { bc->done = 1; return; }
    if (rho == 0.0) { bc->done = 2; return; }
    bc->beta = rho / bc->rho;
    bc->rho = rho;
    if (bc->iters >= bc->maxit) bc->done = 4;
  }
}

// y = x * d (Jacobi scaling); used by the FP32 refinement path
__global__ void __launch_bounds__(kVecThreads) k_mul(const double* __restrict__ x, const double* __restrict__ d,
                                                     double* __restrict__ y, int64_t N) {
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x)
    y[n] = x[n] * d[n];
}

// ----------------------------------------------------------- Richardson
// x <- x + M^-1 r, r = b - A x (Eq. 20), kRichSteps iterations per graph
// launch, each gated on the step counter kstop of the GMRES state, which the
// check kernel lowers (and flags in kdone) once the iteration has stopped.
constexpr int kRichSteps = 8;

// arms the launch's steps, unless an earlier launch stopped (kdone): then the
// launch changes nothing
__global__ void k_rich_begin(GmresDev* gm) { gm->kstop = gm->kdone ? 0 : kRichSteps; }

// x += d * z (Jacobi) or x += z
__global__ void __launch_bounds__(kVecThreads) k_rich_update(double* __restrict__ x, const double* __restrict__ z,
                                                             const double* __restrict__ d, int64_t N,
                                                             const int* kstop, int step) {
  if (kstop && step >= *kstop) return;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x)
    x[n] += d ? d[n] * z[n] : z[n];
}

// r = b - Ax, partials of ||r||^2
__global__ void __launch_bounds__(kVecThreads) k_rich_resid(const double* __restrict__ b,
                                                            const double* __restrict__ Ax, double* __restrict__ r,
                                                            int64_t N, double* __restrict__ part, const int* kstop,
                                                            int step) {
  if (kstop && step >= *kstop) return;
  double s = 0.0;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
    const double v = b[n] - Ax[n];
    r[n] = v;
    s = fma(v, v, s);
  }
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// one warp: rel = ||r|| / ||b||, one more iteration; stop (kstop = step + 1)
// once rel < tol (or is not a number) or the iteration budget is spent
__global__ void k_rich_check(const double* __restrict__ part, int G, GmresDev* gm, double* hist, int hist_cap,
                             int step) {
  if (step >= gm->kstop) return;
  const double s = sum_partials_warp(part, G);
  if (threadIdx.x == 0) {
    const double rel = sqrt(s) / gm->bnorm;
    const int it = gm->iters;
    if (hist && it < hist_cap) hist[it] = rel;
    gm->iters = it + 1;
    gm->rel = rel;
    gm->hist_len = it + 1 < hist_cap ? it + 1 : hist_cap;
    if (!(rel >= gm->tol) || it + 1 >= gm->maxit) {
      gm->kstop = step + 1;
      gm->kdone = 1;   // stopped: the host launches no further graph
    }
  }
}

// y = d * x inside a captured GMRES cycle (skipped once step >= *kstop)
__global__ void __launch_bounds__(kVecThreads) k_mul_gated(const double* __restrict__ x,
                                                           const double* __restrict__ d, double* __restrict__ y,
                                                           int64_t N, const int* kstop, int step) {
  if (kstop && step >= *kstop) return;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x)
    y[n] = x[n] * d[n];
}

}  // namespace


// ------------------------------------------------------------ workspace
struct Workspace {
  double* V;        // (m+1) x N
  double* w[8];     // work vectors
  double* part[2];  // ping-pong partial buffers
};

static rt_status ensure_workspace(Problem* P, int restart, cudaStream_t st) {
  {
    // k_lsq's shared triangle of the longest cycle (103 KB) needs the opt-in;
    // set here, outside any stream capture
    static std::once_flag lsq_attr;
    static cudaError_t lsq_err = cudaSuccess;
    std::call_once(lsq_attr, [] {
      lsq_err = cudaFuncSetAttribute(k_lsq, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lsq_smem(kMaxRestart));
    });
    RT_TRY_CUDA(lsq_err);
  }
  if (!P->vec_grid) {
    int64_t g = (P->Nop + 2 * kVecThreads - 1) / (2 * kVecThreads);
    int cap = 4 * P->num_sms;
    if (cap > kMaxPartials) cap = kMaxPartials;
    P->vec_grid = (int)(g < 1 ? 1 : (g > cap ? cap : g));
  }
  if (!P->work) RT_TRY_CUDA(dev_alloc(P, (void**)&P->work, (size_t)kWorkVecs * P->Nop * sizeof(double)));
  if (!P->dinv) RT_TRY_CUDA(dev_alloc(P, (void**)&P->dinv, (size_t)P->Nop * sizeof(double)));
  if (!P->partials) RT_TRY_CUDA(dev_alloc(P, (void**)&P->partials, (size_t)2 * 2 * kMaxPartials * sizeof(double)));
  if (!P->bpart) RT_TRY_CUDA(dev_alloc(P, (void**)&P->bpart, (size_t)3 * kGramB * kMaxPartials * sizeof(double)));
  if (!P->gm) RT_TRY_CUDA(dev_alloc(P, (void**)&P->gm, sizeof(GmresDev)));
  if (!P->bc) RT_TRY_CUDA(dev_alloc(P, (void**)&P->bc, sizeof(BicgDev)));
  if (restart > P->ws_restart) {
    release_graphs(P);  // captured graphs hold the old basis pointer
    if (P->V) dev_free(P, P->V);
    P->V = nullptr;
    P->ws_restart = 0;
    RT_TRY_CUDA(dev_alloc(P, (void**)&P->V, (size_t)(restart + 1) * P->Nop * sizeof(double)));
    P->ws_restart = restart;
  }
  (void)st;
  return RT_OK;
}

static inline double* wk(Problem* P, int i) { return P->work + (size_t)i * P->Nop; }
static inline double* partb(Problem* P, int i) { return P->partials + (size_t)i * 2 * kMaxPartials; }
// block-pass partials: buffers 0 and 1 ping-pong, 2 holds the Gram partials
static inline double* bpartb(Problem* P, int i) { return P->bpart + (size_t)i * kGramB * kMaxPartials; }

// the dense sigma-form SOR / SSOR preconditioners, and the left ones
static inline bool prec_dense(int pc) {
  return pc == RT_PREC_SOR || pc == RT_PREC_SSOR || pc == RT_PREC_SOR_LEFT || pc == RT_PREC_SSOR_LEFT;
}
static inline bool prec_left(int pc) {
  return pc == RT_PREC_JACOBI_LEFT || pc == RT_PREC_SOR_LEFT || pc == RT_PREC_SSOR_LEFT;
}

// y = M x for a left preconditioner M (D^-1 or the dense P^-1)
static rt_status left_apply(Problem* P, int pc, const double* x, double* y, cudaStream_t st,
                            const int* kstop = nullptr, int step = 0) {
  if (pc == RT_PREC_JACOBI_LEFT) {
    k_mul_gated<<<P->vec_grid, kVecThreads, 0, st>>>(x, P->dinv, y, P->Nop, kstop, step); RT_COUNT(1);
    RT_TRY_CUDA(cudaGetLastError());
    return RT_OK;
  }
  return op_dense_precond_apply(P, x, y, st, kstop, step);
}

// A M^{-1} v with the chosen preconditioner and operator precision
// (nin: GMRES on the I-form; the apply's input v is formed from nin->u, see
// NormIn)
static rt_status apply_prec(Problem* P, const double* v, double* y, int precond, int fp32, cudaStream_t st,
                            const int* kstop = nullptr, int step = 0, const NormIn* nin = nullptr) {
  if (prec_left(precond)) {
    // M A v: the FP64 apply into a scratch vector, then M
    double* t = precond == RT_PREC_JACOBI_LEFT ? P->work + (size_t)6 * P->Nop : P->Mscr + P->Nop;
    RT_TRY(op_apply64(P, v, t, AM_PLAIN, st, kstop, step, nin));
    return left_apply(P, precond, t, y, st, kstop, step);
  }
  if (prec_dense(precond)) {   // right SOR / SSOR: A (P^-1 v)
    RT_TRY(op_dense_precond_apply(P, v, P->Mscr, st, kstop, step));
    return op_apply64(P, P->Mscr, y, AM_PLAIN, st, kstop, step);
  }
  const int mode = precond == RT_PREC_JACOBI ? AM_JACOBI : precond == RT_PREC_LOCAL_LAMBDA ? AM_LOCAL_LAMBDA : AM_PLAIN;
  if (fp32) return op_apply32_f64io(P, v, y, mode, st, kstop, step, nin);
  return op_apply64(P, v, y, mode, st, kstop, step, nin);
}

// x += M^{-1} t  (t may be overwritten)
static rt_status add_precond(Problem* P, double* x, double* t, int precond, double* tmp, cudaStream_t st) {
  const int G = P->vec_grid;
  if (precond == RT_PREC_NONE) {
    k_axpy1<<<G, kVecThreads, 0, st>>>(x, t, P->Nop); RT_COUNT(1);
  } else if (precond == RT_PREC_JACOBI) {
    k_mul<<<G, kVecThreads, 0, st>>>(t, P->dinv, tmp, P->Nop); RT_COUNT(1);
    k_axpy1<<<G, kVecThreads, 0, st>>>(x, tmp, P->Nop); RT_COUNT(1);
  } else if (prec_dense(precond)) {
    RT_TRY(op_dense_precond_apply(P, t, tmp, st));
    k_axpy1<<<G, kVecThreads, 0, st>>>(x, tmp, P->Nop); RT_COUNT(1);
  } else {
    RT_TRY(op_precond_ll(P, t, tmp, st));
    k_axpy1<<<G, kVecThreads, 0, st>>>(x, tmp, P->Nop); RT_COUNT(1);
  }
  RT_TRY_CUDA(cudaGetLastError());
  return RT_OK;
}


// One block-MGS Arnoldi step on w against V[0..j] (see k_bmgs): h_0..h_j
// and h_{j+1} = ||w|| to hcol, v_{j+1} to V, the Gram row j+1 to gram; with
// gm set, the Givens rotations of column j (GMRES).
// scale == false: the normalisation and the fold are left to the next apply
// (NormIn); *pb_out and *ng_out then name the last pass's partial buffer and
// Gram-set count.
static rt_status enqueue_bmgs(Problem* P, double* V, double* w, int j, double* hcol, double* gram, GmresDev* gm,
                              int m, double* hist, int hcap, const int* kstop, cudaStream_t st, bool scale = true,
                              int* pb_out = nullptr, int* ng_out = nullptr) {
  const int Gm = mgs_grid(P);
  const int64_t N = P->Nop;
  using BdotFn = void (*)(const double*, const double*, int64_t, double*, int, int, const int*);
  using BmgsFn = void (*)(double*, const double*, int64_t, int, const double*, double*, double*, const double*, int,
                          int, const int*);
  static const BdotFn bdot[kGramB] = {k_bdot<1>, k_bdot<2>, k_bdot<3>, k_bdot<4>};
  static const BmgsFn pass[kGramB] = {k_bmgs<4, 1>, k_bmgs<4, 2>, k_bmgs<4, 3>, k_bmgs<4, 4>};
  static const BmgsFn last[kGramB] = {k_bmgs<1, 0>, k_bmgs<2, 0>, k_bmgs<3, 0>, k_bmgs<4, 0>};
  static_assert(kGramB == 4, "kernel tables");
  int pb = 0, rev = 0;
  RT_TRY_CUDA(launch_pdl(bdot[std::min(kGramB, j + 1) - 1], Gm, kMgsThreads, st, (const double*)w, (const double*)V, N,
                         bpartb(P, 0), j, rev, kstop)); RT_COUNT(1);
  int ng = 0;
  for (int i0 = 0; i0 <= j; i0 += kGramB) {
    const int nb = std::min(kGramB, j + 1 - i0);
    const int nn = std::max(0, std::min(kGramB, j + 1 - (i0 + nb)));
    if (nn == 0) ng = nb < kGramB ? nb : 0;
    rev ^= 1;
    RT_TRY_CUDA(launch_pdl(nn ? pass[nn - 1] : last[nb - 1], Gm, kMgsThreads, st, w, (const double*)V, N, i0,
                           (const double*)bpartb(P, pb), bpartb(P, pb ^ 1), hcol, (const double*)gram, j, rev,
                           kstop)); RT_COUNT(1);
    pb ^= 1;
  }
  if (pb_out) *pb_out = pb;
  if (ng_out) *ng_out = ng;
  if (!scale) {
    RT_TRY_CUDA(cudaGetLastError());
    return RT_OK;
  }
  rev ^= 1;
  RT_TRY_CUDA(launch_pdl(k_bscale, std::min(Gm, 2 * P->num_sms) + 1, kVecThreads, st, (const double*)w, V, N, (const double*)bpartb(P, pb), Gm, ng,
                         hcol, gram, gm, m, j, hist, hcap, rev, kstop)); RT_COUNT(1);
  RT_TRY_CUDA(cudaGetLastError());
  return RT_OK;
}

// --------------------------------------------------------------- GMRES
struct GmresGraphKey {
  int m, precond, fp32;
  bool operator<(const GmresGraphKey& o) const {
    return std::tie(m, precond, fp32) < std::tie(o.m, o.precond, o.fp32);
  }
};

constexpr int kNumPrec = RT_PREC_SSOR_LEFT + 1;

// bytes of one host copy of a solver's state header (GMRES or BiCGSTAB/CGS)
constexpr size_t kHdrBytes = ((kGmresHeader > sizeof(BicgDev) ? kGmresHeader : sizeof(BicgDev)) + 255) / 256 * 256;

struct GraphCache {
  std::map<GmresGraphKey, cudaGraphExec_t> gmres;
  cudaGraphExec_t bicg[2][kNumPrec][2] = {};  // [method][precond][fp32]
  cudaGraphExec_t rich[kNumPrec] = {};         // [precond]
  std::map<cudaGraphExec_t, long long> kernels;  // kernel nodes per executable graph
  cudaStream_t cap = nullptr;
  // two pinned host copies of the state header and the events that mark
  // them written: the host reads one launch's copy while the next runs
  unsigned char* hdr = nullptr;
  cudaEvent_t hev[2] = {nullptr, nullptr};
  ~GraphCache() {
    if (hdr) cudaFreeHost(hdr);
    for (cudaEvent_t e : hev)
      if (e) cudaEventDestroy(e);
    for (auto& kv : gmres) cudaGraphExecDestroy(kv.second);
    for (auto& a : bicg)
      for (auto& b : a)
        for (auto& c : b)
          if (c) cudaGraphExecDestroy(c);
    for (auto& r : rich)
      if (r) cudaGraphExecDestroy(r);
    if (cap) cudaStreamDestroy(cap);
  }
};

static std::map<const Problem*, GraphCache*>& caches() {
  static std::map<const Problem*, GraphCache*> c;
  return c;
}
static std::mutex g_cache_mu;

static GraphCache* cache_of(Problem* P) {
  std::lock_guard<std::mutex> lk(g_cache_mu);
  auto& c = caches();
  auto it = c.find(P);
  if (it != c.end()) return it->second;
  GraphCache* g = new GraphCache();
  c[P] = g;
  return g;
}

void release_graphs(Problem* P) {
  std::lock_guard<std::mutex> lk(g_cache_mu);
  auto& c = caches();
  auto it = c.find(P);
  if (it != c.end()) {
    delete it->second;
    c.erase(it);
  }
}

// Enqueue one restart cycle: steps 0..m-1, least squares, x update, true
// residual and the start of the next cycle.  Vectors: x = wk(0), b = wk(1),
// r = wk(2), w = wk(3), t = wk(4), Ax = wk(5), tmp = wk(6).
static rt_status enqueue_cycle(Problem* P, int m, int precond, int fp32, cudaStream_t st) {
  const int G = P->vec_grid;
  const int64_t N = P->Nop;
  GmresDev* gm = P->gm;
  const int* kstop = &gm->kstop;
  double* w = wk(P, 3);
  double* hist = P->hist;
  const int hcap = P->hist_cap_dev;
  // I-form: the normalisation of v_{j+1} and the Givens rotations of column
  // j run inside the next step's first operator kernel (NormIn) -- the FP64
  // quadrature, or the FP32 one where the staged FP32 apply takes the
  // basis vectors (a right preconditioner; every v_j shares V's alignment,
  // N being even)
  const int amode = precond == RT_PREC_JACOBI ? AM_JACOBI : precond == RT_PREC_LOCAL_LAMBDA ? AM_LOCAL_LAMBDA : AM_PLAIN;
  const bool fuse = P->form == RT_FORM_I && !prec_dense(precond) &&
                    (!fp32 || (!prec_left(precond) && staged_f64io_ok(P, amode, P->V, w)));
  int pb = 0, ng = 0;
  for (int j = 0; j < m; ++j) {
    double* vj = P->V + (size_t)j * N;
    if (fuse && j > 0) {
      const NormIn nin{w, bpartb(P, pb), mgs_grid(P), ng, &gm->H[(j - 1) * (m + 1)], gm->gram, gm, m, j - 1, hist,
                       hcap, kstop};
      RT_TRY(apply_prec(P, vj, w, precond, fp32, st, kstop, j, &nin));
    } else {
      RT_TRY(apply_prec(P, vj, w, precond, fp32, st, kstop, j));
    }
    // block MGS: dots with the first block, one pass per block of kGramB
    // basis vectors (the last with ||w|| and the Gram dots of v_{j+1}), then
    // (unless fused) the normalisation with the Givens rotations of column j
    RT_TRY(enqueue_bmgs(P, P->V, w, j, &gm->H[j * (m + 1)], gm->gram, gm, m, hist, hcap, kstop, st, !fuse, &pb,
                        &ng));
  }
  if (fuse) {
    k_arnoldi_tail<<<1, 32 * kGramB, 0, st>>>(bpartb(P, pb), mgs_grid(P), ng, &gm->H[(m - 1) * (m + 1)], gm->gram,
                                              gm, m, m - 1, hist, hcap, kstop); RT_COUNT(1);
  }
  RT_TRY_CUDA(cudaGetLastError());
  k_lsq<<<1, 32, lsq_smem(m), st>>>(gm, m); RT_COUNT(1);
  double* x = wk(P, 0);
  double* t = wk(P, 4);
  if (precond == RT_PREC_LOCAL_LAMBDA || precond == RT_PREC_SOR || precond == RT_PREC_SSOR) {
    k_combine<<<G, kVecThreads, 0, st>>>(P->V, N, gm, x, P->dinv, t, 2); RT_COUNT(1);
    if (precond == RT_PREC_LOCAL_LAMBDA) RT_TRY(op_precond_ll(P, t, wk(P, 6), st));
    else RT_TRY(op_dense_precond_apply(P, t, wk(P, 6), st));
    k_axpy1<<<G, kVecThreads, 0, st>>>(x, wk(P, 6), N); RT_COUNT(1);
  } else {
    k_combine<<<G, kVecThreads, 0, st>>>(P->V, N, gm, x, P->dinv, t, precond == RT_PREC_JACOBI ? 1 : 0); RT_COUNT(1);
  }
  RT_TRY(op_apply64(P, x, wk(P, 5), AM_PLAIN, st));
  if (prec_left(precond)) {   // the residual of M A x = M b
    RT_TRY(left_apply(P, precond, wk(P, 5), wk(P, 6), st));
    k_residual<<<G, kVecThreads, 0, st>>>(wk(P, 1), wk(P, 6), wk(P, 2), N, partb(P, 0)); RT_COUNT(1);
  } else {
    k_residual<<<G, kVecThreads, 0, st>>>(wk(P, 1), wk(P, 5), wk(P, 2), N, partb(P, 0)); RT_COUNT(1);
  }
  k_cycle_start<<<G, kVecThreads, 0, st>>>(wk(P, 2), P->V, N, partb(P, 0), gm, m); RT_COUNT(1);
  RT_TRY_CUDA(cudaGetLastError());
  return RT_OK;
}

template <typename F>
static rt_status capture_graph(GraphCache* gc, F&& enqueue, cudaGraphExec_t* out) {
  if (!gc->cap) RT_TRY_CUDA(cudaStreamCreateWithFlags(&gc->cap, cudaStreamNonBlocking));
  RT_TRY_CUDA(cudaStreamBeginCapture(gc->cap, cudaStreamCaptureModeThreadLocal));
  g_capturing = 1;
  rt_status s = enqueue(gc->cap);
  g_capturing = 0;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(gc->cap, &g);
  if (s != RT_OK) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  if (e != cudaSuccess) {
    set_error("graph capture failed: %s", cudaGetErrorString(e));
    return RT_ECUDA;
  }
  size_t nn = 0;
  long long nk = 0;
  if (cudaGraphGetNodes(g, nullptr, &nn) == cudaSuccess && nn) {
    std::vector<cudaGraphNode_t> nodes(nn);
    if (cudaGraphGetNodes(g, nodes.data(), &nn) == cudaSuccess)
      for (size_t i = 0; i < nn; ++i) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++nk;
      }
  }
  cudaGraphExec_t ex = nullptr;
  e = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    set_error("graph instantiate failed: %s", cudaGetErrorString(e));
    return RT_ECUDA;
  }
  gc->kernels[ex] = nk;
  *out = ex;
  return RT_OK;
}

static rt_status launch_graph(GraphCache* gc, cudaGraphExec_t ex, cudaStream_t st) {
  RT_TRY_CUDA(cudaGraphLaunch(ex, st));
  count_launches(gc->kernels[ex]);
  return RT_OK;
}

// Launches `ex` until `stop(header)` holds, one launch ahead of the host:
// launch k+1 and the copy of its state header are queued before the host
// waits for launch k's copy, so the device does not idle while the host
// reads a header and decides.  The graphs this serves leave the state
// unchanged when they run after a stop (their steps are gated off, or they
// repeat a step that changes nothing), so the extra launch queued when the
// stop is seen is waited for and not counted.  `dev` is the header's device
// address, `out` receives the header of the stopping launch; `launches`
// counts the launches up to it.
template <typename Hdr, typename Stop>
static rt_status launch_until(GraphCache* gc, cudaGraphExec_t ex, const Hdr* dev, Hdr* out, size_t bytes,
                              cudaStream_t st, int* launches, Stop&& stop) {
  if (bytes > kHdrBytes) {
    set_error("internal: solver header larger than its host copy");
    return RT_EINVAL;
  }
  if (!gc->hdr) {
    RT_TRY_CUDA(cudaHostAlloc(reinterpret_cast<void**>(&gc->hdr), 2 * kHdrBytes, cudaHostAllocDefault));
    for (cudaEvent_t& e : gc->hev) RT_TRY_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  auto enqueue = [&](int slot) -> rt_status {
    RT_TRY(launch_graph(gc, ex, st));
    RT_TRY_CUDA(cudaMemcpyAsync(gc->hdr + slot * kHdrBytes, dev, bytes, cudaMemcpyDeviceToHost, st));
    RT_TRY_CUDA(cudaEventRecord(gc->hev[slot], st));
    return RT_OK;
  };
  *launches = 0;
  RT_TRY(enqueue(0));
  for (int k = 0;; ++k) {
    const rt_status s = enqueue((k + 1) & 1);   // one ahead
    if (s != RT_OK) {
      cudaStreamSynchronize(st);
      return s;
    }
    RT_TRY_CUDA(cudaEventSynchronize(gc->hev[k & 1]));
    memcpy(static_cast<void*>(out), gc->hdr + (k & 1) * kHdrBytes, bytes);
    *launches += 1;
    if (stop(*out)) break;
  }
  RT_TRY_CUDA(cudaStreamSynchronize(st));   // the launch queued ahead (no effect)
  return RT_OK;
}

static rt_status get_graph(Problem* P, GraphCache* gc, int m, int precond, int fp32, cudaGraphExec_t* out) {
  GmresGraphKey key{m, precond, fp32};
  auto it = gc->gmres.find(key);
  if (it != gc->gmres.end()) {
    *out = it->second;
    return RT_OK;
  }
  cudaGraphExec_t ex = nullptr;
  RT_TRY(capture_graph(gc, [&](cudaStream_t cs) { return enqueue_cycle(P, m, precond, fp32, cs); }, &ex));
  gc->gmres[key] = ex;
  *out = ex;
  return RT_OK;
}

static rt_status ensure_hist(Problem* P, int cap) {
  if (cap > P->hist_cap_dev) {
    if (P->hist) dev_free(P, P->hist);
    P->hist = nullptr;
    P->hist_cap_dev = 0;
    // the graphs bake the history pointer: drop them
    release_graphs(P);
    RT_TRY_CUDA(dev_alloc(P, (void**)&P->hist, (size_t)cap * sizeof(double)));
    P->hist_cap_dev = cap;
  }
  return RT_OK;
}

// Core GMRES on internal buffers: b = wk(1) given, x = wk(0) holds x0 (or
// zero).  Returns the host copy of the final device state.
static rt_status gmres_core(Problem* P, const rt_solver_opts* o, int fp32, double tol, int maxit, bool x0_zero,
                            GmresDev* hs, int* cycles, cudaStream_t st) {
  RT_NVTX("GMRES cycles");
  const int G = P->vec_grid;
  const int64_t N = P->Nop;
  const int m = o->restart;
  std::unique_ptr<GmresDev> initp(new GmresDev);   // large arrays: not on the stack
  GmresDev& init = *initp;
  memset(&init, 0, kGmresHeader);
  init.tol = tol;
  init.maxit = maxit;
  RT_TRY_CUDA(cudaMemcpyAsync(P->gm, &init, kGmresHeader, cudaMemcpyHostToDevice, st));
  RT_TRY_CUDA(cudaStreamSynchronize(st));   // init is freed on return
  k_dot<<<G, kVecThreads, 0, st>>>(wk(P, 1), wk(P, 1), N, partb(P, 1), nullptr, 0, nullptr); RT_COUNT(1);
  k_set_bnorm<<<1, 32, 0, st>>>(partb(P, 1), G, P->gm); RT_COUNT(1);
  if (x0_zero) {
    k_dot<<<G, kVecThreads, 0, st>>>(wk(P, 1), wk(P, 1), N, partb(P, 0), nullptr, 0, nullptr); RT_COUNT(1);
    k_cycle_start<<<G, kVecThreads, 0, st>>>(wk(P, 1), P->V, N, partb(P, 0), P->gm, m); RT_COUNT(1);
  } else {
    RT_TRY(op_apply64(P, wk(P, 0), wk(P, 5), AM_PLAIN, st));
    const double* ax = wk(P, 5);
    if (prec_left(o->precond)) {
      RT_TRY(left_apply(P, o->precond, wk(P, 5), wk(P, 6), st));
      ax = wk(P, 6);
    }
    k_residual<<<G, kVecThreads, 0, st>>>(wk(P, 1), ax, wk(P, 2), N, partb(P, 0)); RT_COUNT(1);
    k_cycle_start<<<G, kVecThreads, 0, st>>>(wk(P, 2), P->V, N, partb(P, 0), P->gm, m); RT_COUNT(1);
  }
  RT_TRY_CUDA(cudaGetLastError());
  RT_TRY_CUDA(cudaMemcpyAsync(hs, P->gm, kGmresHeader, cudaMemcpyDeviceToHost, st));
  RT_TRY_CUDA(cudaStreamSynchronize(st));
  *cycles = 0;
  if (hs->bnorm == 0.0 || !(hs->rel >= tol) || hs->rel != hs->rel) return RT_OK;
  GraphCache* gc = cache_of(P);
  cudaGraphExec_t ex;
  RT_TRY(get_graph(P, gc, m, o->precond, fp32, &ex));
  // A cycle that runs after one of these stops changes nothing: k_cycle_start
  // of the stopping cycle set kstop = 0 (converged, NaN, no steps left), so
  // every step is gated off and the update and residual repeat exactly; or
  // the first step broke down, which the next cycle repeats with the same
  // result (no step done, x unchanged).
  RT_NVTX("GMRES restart cycles (graphs)");
  RT_TRY(launch_until(gc, ex, P->gm, hs, kGmresHeader, st, cycles, [&](const GmresDev& h) {
    return h.rel != h.rel || !(h.rel >= tol) || h.iters >= maxit || (h.breakdown && h.kdone == 0) || h.kstop == 0;
  }));
  return RT_OK;
}

static rt_status prepare(Problem* P, const rt_solver_opts* o, int restart, cudaStream_t st) {
  RT_TRY(ensure_workspace(P, restart, st));
  if (o->resid_hist && o->hist_cap > 0) RT_TRY(ensure_hist(P, o->hist_cap));
  if (o->precond == RT_PREC_JACOBI || o->precond == RT_PREC_JACOBI_LEFT) RT_TRY(op_jacobi_inv(P, P->dinv, st));
  if (o->precond == RT_PREC_JACOBI) RT_TRY(op_jacobi_weights(P, st));
  if (prec_dense(o->precond)) RT_TRY(op_dense_precond_build(P, o->precond, o->omega, st));
  return RT_OK;
}

static rt_status check_opts(const rt_solver_opts* o, const double* b, const double* x) {
  if (!o || !b || !x) { set_error("opts, b_dev and x_dev are required"); return RT_EINVAL; }
  if (o->restart < 1 || o->restart > kMaxRestart) { set_error("restart must be in [1,%d]", kMaxRestart); return RT_EINVAL; }
  if (o->maxit < 1) { set_error("maxit must be >= 1"); return RT_EINVAL; }
  if (o->precond < RT_PREC_NONE || o->precond > RT_PREC_SSOR_LEFT) { set_error("bad precond"); return RT_EINVAL; }
  if (prec_dense(o->precond) && !(o->omega > 0.0 && o->omega < 2.0)) {
    set_error("SOR / SSOR: omega must be in (0, 2)");
    return RT_EINVAL;
  }
  if (prec_dense(o->precond) && o->precision != RT_PRECISION_FP64) {
    set_error("SOR / SSOR need RT_PRECISION_FP64");
    return RT_EINVAL;
  }
  if (o->x0_kind != RT_X0_ZERO && o->x0_kind != RT_X0_USER && o->x0_kind != RT_X0_PAPER) {
    set_error("bad x0_kind");
    return RT_EINVAL;
  }
  if (o->ortho != RT_ORTHO_MGS) { set_error("only RT_ORTHO_MGS is implemented"); return RT_EINVAL; }
  if (o->precision != RT_PRECISION_FP64 && o->precision != RT_PRECISION_FP32_REFINE) { set_error("bad precision"); return RT_EINVAL; }
  if (!(o->rtol > 0.0)) { set_error("rtol must be > 0"); return RT_EINVAL; }
  return RT_OK;
}

static double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

static rt_status finish_info(rt_solve_info* info, rt_status s, double t0) {
  if (info) {
    info->status = s;
    info->t_total_ms = now_ms() - t0;
  }
  return s;
}

// the initial guess into wk(0): zero, the caller's x, or the paper's (Sect. 4.2)
static rt_status load_x0(Problem* P, const rt_solver_opts* o, const double* x, cudaStream_t st) {
  const size_t bytes = (size_t)P->Nop * sizeof(double);
  if (o->x0_kind == RT_X0_USER) RT_TRY_CUDA(cudaMemcpyAsync(wk(P, 0), x, bytes, cudaMemcpyDeviceToDevice, st));
  else if (o->x0_kind == RT_X0_PAPER) RT_TRY(op_x0_paper(P, wk(P, 0), st));
  else RT_TRY_CUDA(cudaMemsetAsync(wk(P, 0), 0, bytes, st));
  return RT_OK;
}

// true relative residual of x = wk(0) against b = wk(1)
static rt_status true_residual(Problem* P, double* rel, cudaStream_t st) {
  RT_NVTX("true residual (FP64 operator)");
  const int G = P->vec_grid;
  RT_TRY(op_apply64(P, wk(P, 0), wk(P, 5), AM_PLAIN, st));
  k_residual<<<G, kVecThreads, 0, st>>>(wk(P, 1), wk(P, 5), wk(P, 2), P->Nop, partb(P, 0)); RT_COUNT(1);
  k_dot<<<G, kVecThreads, 0, st>>>(wk(P, 1), wk(P, 1), P->Nop, partb(P, 1), nullptr, 0, nullptr); RT_COUNT(1);
  RT_TRY_CUDA(cudaGetLastError());
  std::vector<double> h(2 * G);
  RT_TRY_CUDA(cudaMemcpyAsync(h.data(), partb(P, 0), G * sizeof(double), cudaMemcpyDeviceToHost, st));
  RT_TRY_CUDA(cudaMemcpyAsync(h.data() + G, partb(P, 1), G * sizeof(double), cudaMemcpyDeviceToHost, st));
  RT_TRY_CUDA(cudaStreamSynchronize(st));
  double rr = 0, bb = 0;
  for (int i = 0; i < G; ++i) { rr += h[i]; bb += h[G + i]; }
  // a NaN or Inf in b or in the residual gives NaN (RT_ENUMERIC upstream); a
  // zero b gives 0
  if (rr != rr || bb != bb || std::isinf(rr) || std::isinf(bb)) *rel = NAN;
  else *rel = bb > 0 ? sqrt(rr / bb) : 0.0;
  return RT_OK;
}

static rt_status solve_gmres(Problem* P, const rt_solver_opts* o, const double* b, double* x, rt_solve_info* info,
                             cudaStream_t st) {
  const double t0 = now_ms();
  if (info) memset(info, 0, sizeof *info);
  if (prec_left(o->precond) && o->precision != RT_PRECISION_FP64) {
    set_error("the left preconditioners need RT_PRECISION_FP64");
    return finish_info(info, RT_EINVAL, t0);
  }
  RT_TRY(prepare(P, o, o->restart, st));
  const size_t bytes = (size_t)P->Nop * sizeof(double);
  if (prec_left(o->precond)) {   // the system M A x = M b
    RT_TRY(left_apply(P, o->precond, b, wk(P, 1), st));
  } else {
    RT_TRY_CUDA(cudaMemcpyAsync(wk(P, 1), b, bytes, cudaMemcpyDeviceToDevice, st));
  }
  RT_TRY(load_x0(P, o, x, st));
  std::unique_ptr<GmresDev> hsp(new GmresDev);   // only its header is read back
  GmresDev& hs = *hsp;
  int cycles = 0;
  rt_status s = RT_OK;
  int iters = 0, applies = 0, refine = 0;
  double rel = 0.0, est = -1.0;
  if (o->precision == RT_PRECISION_FP64) {
    RT_TRY(gmres_core(P, o, 0, o->rtol, o->maxit, o->x0_kind == RT_X0_ZERO, &hs, &cycles, st));
    iters = hs.iters;
    applies = hs.iters + cycles + (o->x0_kind != RT_X0_ZERO ? 1 : 0);
    rel = hs.bnorm == 0.0 ? 0.0 : hs.rel;
    if (hs.iters > 0 && hs.bnorm != 0.0) est = hs.est;
    if (rel != rel) s = RT_ENUMERIC;
    else if (!(rel < o->rtol) && hs.bnorm != 0.0) s = (hs.breakdown && hs.kdone == 0) ? RT_EBREAKDOWN : RT_ENOTCONV;
  } else {
    // FP32 operator inside FP64 iterative refinement:
    //   r = b - A64 x (FP64);  solve A32 d = r to inner_rtol;  x += d
    // Every restart cycle of the inner GMRES starts from its own FP64
    // residual, so the inner solve refines at each restart by itself; its
    // default tolerance is the outer one (one inner solve normally suffices).
    // No step asks for more than the outer tolerance still needs.
    const double inner0 = o->inner_rtol > 0 ? o->inner_rtol : o->rtol;
    double* xb = wk(P, 7);   // the outer iterate
    RT_TRY_CUDA(cudaMemcpyAsync(xb, wk(P, 0), bytes, cudaMemcpyDeviceToDevice, st));
    double* bsave = wk(P, 8);
    RT_TRY_CUDA(cudaMemcpyAsync(bsave, wk(P, 1), bytes, cudaMemcpyDeviceToDevice, st));
    RT_TRY(true_residual(P, &rel, st));  // r = wk(2)
    applies += 1;
    s = RT_ENOTCONV;
    const int maxref = o->max_refine > 0 ? o->max_refine : 20;
    while (refine < maxref && iters < o->maxit) {
      if (rel != rel) { s = RT_ENUMERIC; break; }
      if (rel < o->rtol) { s = RT_OK; break; }
      RT_NVTX("refinement step");
      // inner solve: b <- r, x <- 0
      RT_TRY_CUDA(cudaMemcpyAsync(wk(P, 1), wk(P, 2), bytes, cudaMemcpyDeviceToDevice, st));
      RT_TRY_CUDA(cudaMemsetAsync(wk(P, 0), 0, bytes, st));
      RT_TRY(gmres_core(P, o, 1, std::max(inner0, o->rtol / rel), o->maxit - iters, true, &hs, &cycles, st));
      if (hs.iters > 0) est = hs.est * rel;   // relative to the inner b = r, which is rel * ||b||
      iters += hs.iters;
      applies += hs.iters + cycles;
      refine += 1;
      k_axpy1<<<P->vec_grid, kVecThreads, 0, st>>>(xb, wk(P, 0), P->Nop); RT_COUNT(1);
      RT_TRY_CUDA(cudaMemcpyAsync(wk(P, 0), xb, bytes, cudaMemcpyDeviceToDevice, st));
      RT_TRY_CUDA(cudaMemcpyAsync(wk(P, 1), bsave, bytes, cudaMemcpyDeviceToDevice, st));
      RT_TRY(true_residual(P, &rel, st));
      applies += 1;
      if (hs.iters == 0) break;
    }
    if (s == RT_ENOTCONV && rel < o->rtol) s = RT_OK;
  }
  RT_TRY_CUDA(cudaMemcpyAsync(x, o->precision == RT_PRECISION_FP64 ? wk(P, 0) : wk(P, 7), bytes,
                              cudaMemcpyDeviceToDevice, st));
  int hl = 0;
  if (o->resid_hist && o->hist_cap > 0 && P->hist) {
    hl = o->precision == RT_PRECISION_FP64 ? hs.hist_len : 0;
    if (hl > o->hist_cap) hl = o->hist_cap;
    if (hl) RT_TRY_CUDA(cudaMemcpyAsync(o->resid_hist, P->hist, hl * sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  RT_TRY_CUDA(cudaStreamSynchronize(st));
  if (o->precision == RT_PRECISION_FP32_REFINE) {
    const rt_status f = check_device_flag(P, st);
    if (f != RT_OK) s = f;
  }
  if (info) {
    info->iters = iters;
    info->restarts = cycles;
    info->applies = applies;
    info->refine_steps = refine;
    info->rel_resid = rel;
    info->err_est = est >= 0.0 ? est : rel;
    info->hist_len = hl;
  }
  return finish_info(info, s, t0);
}

// ----------------------------------------------------------- BiCGSTAB / CGS
// vectors: x0 = wk(0), b = wk(1), r = wk(2), rhat = wk(3), p = wk(4),
// v = wk(5), s = wk(6), t = wk(7) (BiCGSTAB);  CGS: u = wk(5), q = wk(6),
// w/vhat = wk(7) and V[0], V[1] as scratch.  acc = V[2] accumulates the
// unpreconditioned direction sum; x = x0 + M^{-1} acc at the end.
static rt_status enqueue_bicg_iter(Problem* P, int method, int precond, int fp32, cudaStream_t st) {
  const int G = P->vec_grid;
  const int64_t N = P->Nop;
  BicgDev* bc = P->bc;
  double* acc = P->V + 2 * (size_t)N;
  double *r = wk(P, 2), *rhat = wk(P, 3), *p = wk(P, 4);
  if (method == 0) {
    double *v = wk(P, 5), *s = wk(P, 6), *t = wk(P, 7);
    k_bs_p<<<G, kVecThreads, 0, st>>>(p, r, v, N, bc); RT_COUNT(1);
    RT_TRY(apply_prec(P, p, v, precond, fp32, st));
    k_dot<<<G, kVecThreads, 0, st>>>(rhat, v, N, partb(P, 0), nullptr, 0, &bc->done); RT_COUNT(1);
    k_bc_alpha<<<1, 32, 0, st>>>(bc, partb(P, 0), G); RT_COUNT(1);
    k_bs_s<<<G, kVecThreads, 0, st>>>(s, r, v, N, bc, partb(P, 1)); RT_COUNT(1);
    k_bs_check_s<<<1, 32, 0, st>>>(bc, partb(P, 1), G); RT_COUNT(1);
    RT_TRY(apply_prec(P, s, t, precond, fp32, st));
    k_dot2<<<G, kVecThreads, 0, st>>>(t, s, t, t, N, partb(P, 0), &bc->done); RT_COUNT(1);
    k_bs_omega<<<1, 32, 0, st>>>(bc, partb(P, 0), G); RT_COUNT(1);
    k_bs_update<<<G, kVecThreads, 0, st>>>(acc, p, s, t, r, rhat, N, bc, partb(P, 1)); RT_COUNT(1);
    k_bs_check_r<<<1, 32, 0, st>>>(bc, partb(P, 1), G, P->hist, P->hist_cap_dev); RT_COUNT(1);
  } else {
    double *u = wk(P, 5), *q = wk(P, 6), *w = wk(P, 7);
    double* vh = P->V;
    double* qh = P->V + (size_t)N;
    k_cgs_up<<<G, kVecThreads, 0, st>>>(u, p, r, q, N, bc); RT_COUNT(1);
    RT_TRY(apply_prec(P, p, vh, precond, fp32, st));
    k_dot<<<G, kVecThreads, 0, st>>>(rhat, vh, N, partb(P, 0), nullptr, 0, &bc->done); RT_COUNT(1);
    k_bc_alpha<<<1, 32, 0, st>>>(bc, partb(P, 0), G); RT_COUNT(1);
    k_cgs_q<<<G, kVecThreads, 0, st>>>(q, w, acc, u, vh, N, bc); RT_COUNT(1);
    RT_TRY(apply_prec(P, w, qh, precond, fp32, st));
    k_cgs_r<<<G, kVecThreads, 0, st>>>(r, qh, rhat, N, bc, partb(P, 1)); RT_COUNT(1);
    k_cgs_check<<<1, 32, 0, st>>>(bc, partb(P, 1), G, P->hist, P->hist_cap_dev); RT_COUNT(1);
  }
  RT_TRY_CUDA(cudaGetLastError());
  return RT_OK;
}

// a kernel that skips when done: apply_prec launches operator kernels that do
// not look at the flag, so an iteration after convergence still computes an
// (unused) product; the graph therefore holds one iteration and the host
// checks the flag after every launch (one launch behind the device,
// launch_until).
// Richardson iterations of one graph launch: vectors x = wk(0), b = wk(1),
// r = wk(2), Ax = wk(5), z = wk(6)
static rt_status enqueue_rich(Problem* P, int precond, cudaStream_t st) {
  const int G = P->vec_grid;
  const int64_t N = P->Nop;
  GmresDev* gm = P->gm;
  const int* kstop = &gm->kstop;
  k_rich_begin<<<1, 1, 0, st>>>(gm); RT_COUNT(1);
  for (int s = 0; s < kRichSteps; ++s) {
    if (precond == RT_PREC_LOCAL_LAMBDA || prec_dense(precond)) {
      if (precond == RT_PREC_LOCAL_LAMBDA) RT_TRY(op_precond_ll(P, wk(P, 2), wk(P, 6), st, kstop, s));
      else RT_TRY(op_dense_precond_apply(P, wk(P, 2), wk(P, 6), st, kstop, s));
      k_rich_update<<<G, kVecThreads, 0, st>>>(wk(P, 0), wk(P, 6), nullptr, N, kstop, s); RT_COUNT(1);
    } else {
      k_rich_update<<<G, kVecThreads, 0, st>>>(wk(P, 0), wk(P, 2), precond == RT_PREC_JACOBI ? P->dinv : nullptr, N,
                                               kstop, s); RT_COUNT(1);
    }
    RT_TRY(op_apply64(P, wk(P, 0), wk(P, 5), AM_PLAIN, st, kstop, s));
    k_rich_resid<<<G, kVecThreads, 0, st>>>(wk(P, 1), wk(P, 5), wk(P, 2), N, partb(P, 0), kstop, s); RT_COUNT(1);
    k_rich_check<<<1, 32, 0, st>>>(partb(P, 0), G, gm, P->hist, P->hist_cap_dev, s); RT_COUNT(1);
  }
  RT_TRY_CUDA(cudaGetLastError());
  return RT_OK;
}

static rt_status solve_richardson(Problem* P, const rt_solver_opts* o, const double* b, double* x,
                                  rt_solve_info* info, cudaStream_t st) {
  const double t0 = now_ms();
  if (info) memset(info, 0, sizeof *info);
  if (o->precision != RT_PRECISION_FP64 || prec_left(o->precond)) {
    set_error("Richardson: FP64, with NONE, JACOBI, LOCAL_LAMBDA, SOR or SSOR");
    return finish_info(info, RT_EINVAL, t0);
  }
  RT_TRY(prepare(P, o, 1, st));
  const int G = P->vec_grid;
  const int64_t N = P->Nop;
  const size_t bytes = (size_t)N * sizeof(double);
  RT_TRY_CUDA(cudaMemcpyAsync(wk(P, 1), b, bytes, cudaMemcpyDeviceToDevice, st));
  int applies = 0;
  if (o->x0_kind != RT_X0_ZERO) {
    RT_TRY(load_x0(P, o, x, st));
    RT_TRY(op_apply64(P, wk(P, 0), wk(P, 5), AM_PLAIN, st));
    k_residual<<<G, kVecThreads, 0, st>>>(wk(P, 1), wk(P, 5), wk(P, 2), N, partb(P, 0)); RT_COUNT(1);
    applies = 1;
  } else {
    RT_TRY_CUDA(cudaMemsetAsync(wk(P, 0), 0, bytes, st));
    RT_TRY_CUDA(cudaMemcpyAsync(wk(P, 2), b, bytes, cudaMemcpyDeviceToDevice, st));
    k_dot<<<G, kVecThreads, 0, st>>>(wk(P, 2), wk(P, 2), N, partb(P, 0), nullptr, 0, nullptr); RT_COUNT(1);
  }
  k_dot<<<G, kVecThreads, 0, st>>>(wk(P, 1), wk(P, 1), N, partb(P, 1), nullptr, 0, nullptr); RT_COUNT(1);
  RT_TRY_CUDA(cudaGetLastError());
  std::vector<double> h(2 * G);
  RT_TRY_CUDA(cudaMemcpyAsync(h.data(), partb(P, 0), G * sizeof(double), cudaMemcpyDeviceToHost, st));
  RT_TRY_CUDA(cudaMemcpyAsync(h.data() + G, partb(P, 1), G * sizeof(double), cudaMemcpyDeviceToHost, st));
  RT_TRY_CUDA(cudaStreamSynchronize(st));
  double rr = 0, bb = 0;
  for (int i = 0; i < G; ++i) { rr += h[i]; bb += h[G + i]; }
  std::unique_ptr<GmresDev> hsp(new GmresDev);
  GmresDev& hs = *hsp;
  memset(&hs, 0, kGmresHeader);
  hs.bnorm = sqrt(bb);
  hs.tol = o->rtol;
  hs.maxit = o->maxit;
  // NaN or Inf in b or x0 gives NaN (RT_ENUMERIC below); a zero b gives 0
  if (rr != rr || bb != bb || std::isinf(rr) || std::isinf(bb)) hs.rel = NAN;
  else hs.rel = hs.bnorm > 0.0 ? sqrt(rr) / hs.bnorm : 0.0;
  rt_status s = RT_OK;
  if (hs.bnorm > 0.0 && hs.rel >= o->rtol) {
    RT_TRY_CUDA(cudaMemcpyAsync(P->gm, &hs, kGmresHeader, cudaMemcpyHostToDevice, st));
    GraphCache* gc = cache_of(P);
    cudaGraphExec_t& ex = gc->rich[o->precond];
    if (!ex) {
      const int prec = o->precond;
      RT_TRY(capture_graph(gc, [&](cudaStream_t cs) { return enqueue_rich(P, prec, cs); }, &ex));
    }
    RT_NVTX("Richardson iterations (graphs)");
    int launches = 0;
    RT_TRY(launch_until(gc, ex, P->gm, &hs, kGmresHeader, st, &launches,
                        [](const GmresDev& h) { return h.kdone != 0; }));   // stopped inside this launch
  } else if (hs.bnorm == 0.0) {
    RT_TRY_CUDA(cudaMemsetAsync(wk(P, 0), 0, bytes, st));
    hs.rel = 0.0;
  }
  if (hs.rel != hs.rel) s = RT_ENUMERIC;
  else if (!(hs.rel < o->rtol) && hs.bnorm > 0.0) s = RT_ENOTCONV;
  RT_TRY_CUDA(cudaMemcpyAsync(x, wk(P, 0), bytes, cudaMemcpyDeviceToDevice, st));
  int hl = 0;
  if (o->resid_hist && o->hist_cap > 0 && P->hist) {
    hl = hs.iters < o->hist_cap ? hs.iters : o->hist_cap;
    if (hl) RT_TRY_CUDA(cudaMemcpyAsync(o->resid_hist, P->hist, hl * sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  RT_TRY_CUDA(cudaStreamSynchronize(st));
  if (info) {
    info->iters = hs.iters;
    info->applies = applies + hs.iters;
    info->rel_resid = hs.rel;
    info->err_est = hs.rel;   // every step forms the FP64 residual itself
    info->hist_len = hl;
  }
  return finish_info(info, s, t0);
}

// BiCGSTAB (method 0) or CGS (method 1) on the internal buffers: b = wk(1);
// x0 = wk(0) (set to zero here when x0_zero); fp32 selects the FP32 operator.
// On return wk(0) = x0 + M^{-1} acc, *hs holds the final device state and
// *applies counts the products with A; *zero_b is set when ||b|| = 0 (x = 0).
static rt_status bicg_core(Problem* P, int method, const rt_solver_opts* o, int fp32, double tol, int maxit,
                           bool x0_zero, BicgDev* hs, int* applies, bool* zero_b, cudaStream_t st) {
  const int G = P->vec_grid;
  const int64_t N = P->Nop;
  const size_t bytes = (size_t)N * sizeof(double);
  double *x0 = wk(P, 0), *bb = wk(P, 1), *r = wk(P, 2), *rhat = wk(P, 3);
  double* acc = P->V + 2 * (size_t)N;
  *zero_b = false;
  if (!x0_zero) {
    RT_TRY(op_apply64(P, x0, wk(P, 5), AM_PLAIN, st));
    k_residual<<<G, kVecThreads, 0, st>>>(bb, wk(P, 5), r, N, partb(P, 0)); RT_COUNT(1);
    *applies += 1;
  } else {
    RT_TRY_CUDA(cudaMemsetAsync(x0, 0, bytes, st));
    RT_TRY_CUDA(cudaMemcpyAsync(r, bb, bytes, cudaMemcpyDeviceToDevice, st));
  }
  RT_TRY_CUDA(cudaMemcpyAsync(rhat, r, bytes, cudaMemcpyDeviceToDevice, st));
  for (int i = 4; i < 8; ++i) RT_TRY_CUDA(cudaMemsetAsync(wk(P, i), 0, bytes, st));
  RT_TRY_CUDA(cudaMemsetAsync(acc, 0, bytes, st));
  BicgDev init;
  memset(&init, 0, sizeof init);
  init.tol = tol;
  init.maxit = maxit;
  RT_TRY_CUDA(cudaMemcpyAsync(P->bc, &init, sizeof init, cudaMemcpyHostToDevice, st));
  // ||b||, then ||r||^2 and <rhat, r>
  k_dot<<<G, kVecThreads, 0, st>>>(bb, bb, N, partb(P, 1), nullptr, 0, nullptr); RT_COUNT(1);
  k_dot2<<<G, kVecThreads, 0, st>>>(r, r, rhat, r, N, partb(P, 0), nullptr); RT_COUNT(1);
  RT_TRY_CUDA(cudaGetLastError());
  {
    std::vector<double> h(G);
    RT_TRY_CUDA(cudaMemcpyAsync(h.data(), partb(P, 1), G * sizeof(double), cudaMemcpyDeviceToHost, st));
    RT_TRY_CUDA(cudaStreamSynchronize(st));
    double s2 = 0;
    for (int i = 0; i < G; ++i) s2 += h[i];
    init.bnorm = sqrt(s2);
    if (init.bnorm == 0.0) {
      RT_TRY_CUDA(cudaMemsetAsync(x0, 0, bytes, st));
      *zero_b = true;
      memset(hs, 0, sizeof *hs);
      hs->done = 1;
      return RT_OK;
    }
    RT_TRY_CUDA(cudaMemcpyAsync(&P->bc->bnorm, &init.bnorm, sizeof(double), cudaMemcpyHostToDevice, st));
  }
  k_bc_init<<<1, 32, 0, st>>>(P->bc, partb(P, 0), G); RT_COUNT(1);
  RT_TRY_CUDA(cudaGetLastError());
  GraphCache* gc = cache_of(P);
  cudaGraphExec_t& ex = gc->bicg[method][o->precond][fp32 ? 1 : 0];
  if (!ex) {
    const int prec = o->precond;
    RT_TRY(capture_graph(gc, [&](cudaStream_t cs) { return enqueue_bicg_iter(P, method, prec, fp32, cs); }, &ex));
  }
  RT_TRY_CUDA(cudaMemcpyAsync(hs, P->bc, sizeof *hs, cudaMemcpyDeviceToHost, st));
  RT_TRY_CUDA(cudaStreamSynchronize(st));
  if (!hs->done) {
    // An iteration after the stop changes nothing: its vector kernels skip
    // (the half-step update is applied once, marked by half = 2) and its
    // operator products are recomputed from unchanged inputs.
    RT_NVTX("BiCGSTAB/CGS iterations (graphs)");
    int its = 0;
    RT_TRY(launch_until(gc, ex, P->bc, hs, sizeof *hs, st, &its, [&](const BicgDev& h) {
      *applies += h.half ? 1 : 2;
      return h.done != 0;
    }));
  }
  // x = x0 + M^{-1} acc
  RT_TRY(add_precond(P, x0, acc, o->precond, wk(P, 6), st));
  return RT_OK;
}

static rt_status bicg_status(const BicgDev& hs) {
  return hs.done == 1 ? RT_OK : hs.done == 2 ? RT_EBREAKDOWN : hs.done == 3 ? RT_ENUMERIC : RT_ENOTCONV;
}

static rt_status solve_bicg(Problem* P, int method, const rt_solver_opts* o, const double* b, double* x,
                            rt_solve_info* info, cudaStream_t st) {
  const double t0 = now_ms();
  if (info) memset(info, 0, sizeof *info);
  if (prec_left(o->precond)) {
    set_error("BiCGSTAB/CGS are preconditioned from the right only");
    return finish_info(info, RT_EINVAL, t0);
  }
  const bool refine = o->precision == RT_PRECISION_FP32_REFINE;
  // two more basis-sized vectors for the refinement: the outer iterate and b
  RT_TRY(prepare(P, o, refine ? 4 : 2, st));
  const int64_t N = P->Nop;
  const size_t bytes = (size_t)N * sizeof(double);
  RT_TRY_CUDA(cudaMemcpyAsync(wk(P, 1), b, bytes, cudaMemcpyDeviceToDevice, st));
  if (o->x0_kind != RT_X0_ZERO) RT_TRY(load_x0(P, o, x, st));
  int applies = 0, iters = 0, refine_steps = 0;
  BicgDev hs;
  memset(&hs, 0, sizeof hs);
  bool zero_b = false;
  rt_status s = RT_OK;
  double rel = 0, est = -1.0;
  if (!refine) {
    RT_TRY(bicg_core(P, method, o, 0, o->rtol, o->maxit, o->x0_kind == RT_X0_ZERO, &hs, &applies, &zero_b, st));
    iters = hs.iters;
    if (zero_b) {
      RT_TRY_CUDA(cudaMemsetAsync(x, 0, bytes, st));
      RT_TRY_CUDA(cudaStreamSynchronize(st));
      if (info) info->rel_resid = info->err_est = 0.0;
      return finish_info(info, RT_OK, t0);
    }
    s = bicg_status(hs);
    est = hs.rel;   // the recursively updated residual
    RT_TRY_CUDA(cudaMemcpyAsync(x, wk(P, 0), bytes, cudaMemcpyDeviceToDevice, st));
    RT_TRY(true_residual(P, &rel, st));
  } else {
    // FP32 operator inside FP64 iterative refinement, as for GMRES:
    //   r = b - A64 x (FP64);  solve A32 d = r to inner_rtol;  x += d
    // The inner iteration never forms the FP64 residual, so its default
    // tolerance is 1e-4; no step asks for more than the outer tolerance
    // still needs.
    const double inner0 = o->inner_rtol > 0 ? o->inner_rtol : 1e-4;
    double* xb = P->V + 3 * (size_t)N;    // the outer iterate
    double* bsave = P->V + 4 * (size_t)N;
    if (o->x0_kind == RT_X0_ZERO) RT_TRY_CUDA(cudaMemsetAsync(wk(P, 0), 0, bytes, st));
    RT_TRY_CUDA(cudaMemcpyAsync(xb, wk(P, 0), bytes, cudaMemcpyDeviceToDevice, st));
    RT_TRY_CUDA(cudaMemcpyAsync(bsave, wk(P, 1), bytes, cudaMemcpyDeviceToDevice, st));
    RT_TRY(true_residual(P, &rel, st));   // r = wk(2)
    applies += 1;
    s = RT_ENOTCONV;
    const int maxref = o->max_refine > 0 ? o->max_refine : 20;
    while (refine_steps < maxref && iters < o->maxit) {
      if (rel != rel) { s = RT_ENUMERIC; break; }
      if (rel < o->rtol) { s = RT_OK; break; }
      RT_NVTX("refinement step");
      RT_TRY_CUDA(cudaMemcpyAsync(wk(P, 1), wk(P, 2), bytes, cudaMemcpyDeviceToDevice, st));
      RT_TRY(bicg_core(P, method, o, 1, std::max(inner0, o->rtol / rel), o->maxit - iters, true, &hs, &applies,
                       &zero_b, st));
      iters += hs.iters;
      refine_steps += 1;
      const rt_status inner = bicg_status(hs);
      if (inner == RT_EBREAKDOWN && hs.iters == 0) { s = RT_EBREAKDOWN; break; }
      // x + d into wk(0); keep it only if the FP64 residual went down (an
      // inner solve that failed with the FP32 operator must not spoil x)
      k_axpy1<<<P->vec_grid, kVecThreads, 0, st>>>(wk(P, 0), xb, N); RT_COUNT(1);
      RT_TRY_CUDA(cudaMemcpyAsync(wk(P, 1), bsave, bytes, cudaMemcpyDeviceToDevice, st));
      const double prev = rel;
      RT_TRY(true_residual(P, &rel, st));
      applies += 1;
      est = hs.rel * prev;   // the inner estimate, relative to its b = r (prev * ||b||)
      if (!(rel < prev)) {   // rejected: x stays the last accepted iterate, with its residual
        rel = prev;
        est = prev;
        s = (inner == RT_ENUMERIC || hs.done == 3) ? RT_ENUMERIC : RT_ENOTCONV;
        break;
      }
      RT_TRY_CUDA(cudaMemcpyAsync(xb, wk(P, 0), bytes, cudaMemcpyDeviceToDevice, st));
      if (hs.iters == 0) break;
    }
    if (rel != rel) s = RT_ENUMERIC;
    else if (s == RT_ENOTCONV && rel < o->rtol) s = RT_OK;
    RT_TRY_CUDA(cudaMemcpyAsync(x, xb, bytes, cudaMemcpyDeviceToDevice, st));
  }
  int hl = 0;
  if (o->resid_hist && o->hist_cap > 0 && P->hist) {
    hl = hs.iters < o->hist_cap ? hs.iters : o->hist_cap;
    if (hl) RT_TRY_CUDA(cudaMemcpyAsync(o->resid_hist, P->hist, hl * sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  RT_TRY_CUDA(cudaStreamSynchronize(st));
  if (info) {
    info->iters = iters;
    info->applies = applies;
    info->refine_steps = refine_steps;
    info->rel_resid = rel;
    info->err_est = est >= 0.0 && est == est ? est : rel;
    info->hist_len = hl;
  }
  return finish_info(info, s, t0);
}

}  // namespace rt

using namespace rt;

extern "C" {

void rt_solver_opts_default(rt_solver_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof *o);
  o->restart = 30;
  o->maxit = 10000;
  o->precond = RT_PREC_JACOBI;
  o->x0_kind = RT_X0_ZERO;
  o->ortho = RT_ORTHO_MGS;
  o->precision = RT_PRECISION_FP64;
  o->rtol = 1e-8;
  o->inner_rtol = 0.0;   // per solver: GMRES rtol, BiCGSTAB/CGS 1e-4
  o->max_refine = 20;
  o->omega = 1.0;
}

rt_status rt_arnoldi_mgs(rt_problem* prob, double* V_dev, int32_t j, double* w_dev, double* h_dev, void* stream) {
  RT_NVTX("rt_arnoldi_mgs");
  clear_error();
  if (!prob || !V_dev || !w_dev || !h_dev) { set_error("prob, V_dev, w_dev and h_dev are required"); return RT_EINVAL; }
  if (j < 0 || j >= kMaxRestart) { set_error("j must be in [0,%d)", kMaxRestart); return RT_EINVAL; }
  Problem* P = &prob->P;
  cudaStream_t st = as_stream(stream);
  RT_TRY(ensure_workspace(P, 1, st));
  const int G = P->vec_grid;
  const int64_t N = P->Nop;
  // the kernels gate on kstop: point it at a device int that never stops them
  int* always = reinterpret_cast<int*>(&P->gm->kstop);
  const int big = 1 << 30;
  RT_TRY_CUDA(cudaMemcpyAsync(always, &big, sizeof(int), cudaMemcpyHostToDevice, st));
  int pb = 0;
  k_dot<<<G, kVecThreads, 0, st>>>(w_dev, V_dev, N, partb(P, pb), nullptr, 0, nullptr); RT_COUNT(1);
  for (int i = 0; i <= j; ++i) {
    const double* vprev = V_dev + (size_t)i * N;
    const double* vnext = (i < j) ? V_dev + (size_t)(i + 1) * N : nullptr;
    k_mgs<<<G, kVecThreads, 0, st>>>(w_dev, vprev, vnext, N, partb(P, pb), partb(P, pb ^ 1), h_dev + i, always, 0); RT_COUNT(1);
    pb ^= 1;
  }
  k_norm_out<<<G, kVecThreads, 0, st>>>(w_dev, V_dev + (size_t)(j + 1) * N, N, partb(P, pb), h_dev + j + 1); RT_COUNT(1);
  RT_TRY_CUDA(cudaGetLastError());
  return RT_OK;
}

rt_status rt_arnoldi_bmgs(rt_problem* prob, double* V_dev, int32_t j, double* w_dev, double* gram_dev,
                          double* h_dev, void* stream) {
  RT_NVTX("rt_arnoldi_bmgs");
  clear_error();
  if (!prob || !V_dev || !w_dev || !gram_dev || !h_dev) {
    set_error("prob, V_dev, w_dev, gram_dev and h_dev are required");
    return RT_EINVAL;
  }
  if (j < 0 || j >= kMaxRestart) { set_error("j must be in [0,%d)", kMaxRestart); return RT_EINVAL; }
  Problem* P = &prob->P;
  cudaStream_t st = as_stream(stream);
  RT_TRY(ensure_workspace(P, 1, st));
  int* always = reinterpret_cast<int*>(&P->gm->kstop);   // a gate that never stops the kernels
  const int big = 1 << 30;
  RT_TRY_CUDA(cudaMemcpyAsync(always, &big, sizeof(int), cudaMemcpyHostToDevice, st));
  return enqueue_bmgs(P, V_dev, w_dev, j, h_dev, gram_dev, nullptr, 0, nullptr, 0, always, st);
}

rt_status rt_solve_gmres(rt_problem* prob, const rt_solver_opts* opts, const double* b_dev, double* x_dev,
                         rt_solve_info* info, void* stream) {
  RT_NVTX("rt_solve_gmres");
  clear_error();
  if (!prob) { set_error("prob is NULL"); return RT_EINVAL; }
  RT_TRY(check_opts(opts, b_dev, x_dev));
  return solve_gmres(&prob->P, opts, b_dev, x_dev, info, as_stream(stream));
}

rt_status rt_solve_bicgstab(rt_problem* prob, const rt_solver_opts* opts, const double* b_dev, double* x_dev,
                            rt_solve_info* info, void* stream) {
  RT_NVTX("rt_solve_bicgstab");
  clear_error();
  if (!prob) { set_error("prob is NULL"); return RT_EINVAL; }
  RT_TRY(check_opts(opts, b_dev, x_dev));
  return solve_bicg(&prob->P, 0, opts, b_dev, x_dev, info, as_stream(stream));
}

rt_status rt_solve_cgs(rt_problem* prob, const rt_solver_opts* opts, const double* b_dev, double* x_dev,
                       rt_solve_info* info, void* stream) {
  RT_NVTX("rt_solve_cgs");
  clear_error();
  if (!prob) { set_error("prob is NULL"); return RT_EINVAL; }
  RT_TRY(check_opts(opts, b_dev, x_dev));
  return solve_bicg(&prob->P, 1, opts, b_dev, x_dev, info, as_stream(stream));
}

rt_status rt_solve_richardson(rt_problem* prob, const rt_solver_opts* opts, const double* b_dev, double* x_dev,
                              rt_solve_info* info, void* stream) {
  RT_NVTX("rt_solve_richardson");
  clear_error();
  if (!prob) { set_error("prob is NULL"); return RT_EINVAL; }
  RT_TRY(check_opts(opts, b_dev, x_dev));
  return solve_richardson(&prob->P, opts, b_dev, x_dev, info, as_stream(stream));
}

}  // extern "C"

// ---------------------------------------------------------------------------
// MGS Arnoldi step without device allocation.
//
// For callers that cannot call cudaMalloc: code running while a CUDA stream is
// being captured into a graph, processes whose device memory is entirely owned
// by another allocator that must account for every byte, and service loops
// where the device-wide synchronisation an allocation may cause is not
// acceptable.  The only scratch this step needs -- one deterministic partial
// sum per block for each reduction -- lives in the file-scope array below,
// which every GPU that loads the library keeps until the process exits.
namespace rt {
namespace {
constexpr int kStaticPartials = 1024;   // partial sums per reduction (blocks of the grid)
static __device__ __align__(256) double g_static_scratch[2 * kStaticPartials];
static __device__ int g_static_never_stop = 1 << 30;   // gate value for k_mgs: never skip

struct StaticScratch {
  double* scratch = nullptr;
  int* gate = nullptr;
  int grid_cap = 0;
};
std::mutex g_static_mu;
std::map<unsigned long long, StaticScratch> g_static_by_context;

// Identity of the current device's context: the driver's per-context id,
// unique for the life of the process, so a context created after a device
// reset (which reloads the module and moves the array) gets a new entry.
// Before the context exists (first call in a process), or where the driver
// does not offer the id, the device ordinal is used; cudaGetSymbolAddress
// then creates the context, and later calls key on its id (one more lookup).
using PfnCtxGetCurrent = CUresult (*)(CUcontext*);
using PfnCtxGetId = CUresult (*)(CUcontext, unsigned long long*);
unsigned long long current_context_key(int dev) {
  static PfnCtxGetCurrent get_current = nullptr;
  static PfnCtxGetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<PfnCtxGetCurrent>(fn);
    fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<PfnCtxGetId>(fn);
  });
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (get_current && get_id && get_current(&ctx) == CUDA_SUCCESS && ctx && get_id(ctx, &id) == CUDA_SUCCESS)
    return id;
  return (1ull << 63) | (unsigned long long)dev;
}

// Device addresses of the static scratch in the current device's context;
// looked up once per context (cudaGetSymbolAddress, with the device current)
// and cached.
rt_status static_scratch_for_current_device(StaticScratch* out) {
  int dev = 0;
  RT_TRY_CUDA(cudaGetDevice(&dev));
  const unsigned long long key = current_context_key(dev);
  std::lock_guard<std::mutex> lk(g_static_mu);
  auto it = g_static_by_context.find(key);
  if (it == g_static_by_context.end()) {
    StaticScratch s;
    RT_TRY_CUDA(cudaGetSymbolAddress((void**)&s.scratch, g_static_scratch));
    RT_TRY_CUDA(cudaGetSymbolAddress((void**)&s.gate, g_static_never_stop));
    int sms = 0;
    RT_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    s.grid_cap = 4 * sms < kStaticPartials ? 4 * sms : kStaticPartials;
    it = g_static_by_context.emplace(key, s).first;
  }
  *out = it->second;
  return RT_OK;
}
}  // namespace
}  // namespace rt

extern "C" {

rt_status rt_arnoldi_mgs_static(double* V_dev, int64_t N, int32_t j, double* w_dev, double* h_dev, void* stream) {
  RT_NVTX("rt_arnoldi_mgs_static");
  clear_error();
  if (!V_dev || !w_dev || !h_dev) { set_error("V_dev, w_dev and h_dev are required"); return RT_EINVAL; }
  if (N < 1 || N > RT_ARNOLDI_STATIC_MAX_N) {
    set_error("N must be in [1, %lld] (got %lld)", (long long)RT_ARNOLDI_STATIC_MAX_N, (long long)N);
    return RT_EINVAL;
  }
  if (j < 0 || j >= RT_ARNOLDI_STATIC_MAX_J) {
    set_error("j must be in [0, %d) (got %d)", RT_ARNOLDI_STATIC_MAX_J, (int)j);
    return RT_EINVAL;
  }
  StaticScratch sc;
  RT_TRY(static_scratch_for_current_device(&sc));
  cudaStream_t st = as_stream(stream);
  int64_t g = (N + 2 * kVecThreads - 1) / (2 * kVecThreads);
  const int G = (int)(g < 1 ? 1 : (g > sc.grid_cap ? sc.grid_cap : g));
  double* part[2] = {sc.scratch, sc.scratch + kStaticPartials};
  // every partial a kernel reads was written earlier in this call by the
  // kernel before it, for the same grid size: nothing has to start at zero
  int pb = 0;
  k_dot<<<G, kVecThreads, 0, st>>>(w_dev, V_dev, N, part[pb], nullptr, 0, nullptr); RT_COUNT(1);
  for (int i = 0; i <= j; ++i) {
    const double* vprev = V_dev + (size_t)i * N;
    const double* vnext = (i < j) ? V_dev + (size_t)(i + 1) * N : nullptr;
    k_mgs<<<G, kVecThreads, 0, st>>>(w_dev, vprev, vnext, N, part[pb], part[pb ^ 1], h_dev + i, sc.gate, 0); RT_COUNT(1);
    pb ^= 1;
  }
  k_norm_out<<<G, kVecThreads, 0, st>>>(w_dev, V_dev + (size_t)(j + 1) * N, N, part[pb], h_dev + j + 1); RT_COUNT(1);
  RT_TRY_CUDA(cudaGetLastError());
  return RT_OK;
}

}  // extern "C"

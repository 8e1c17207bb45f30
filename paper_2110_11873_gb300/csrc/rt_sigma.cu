// The sigma-form system of Eq. (18) on the device (FP64): the unknown is
// sigma = (sigma^0_0(k), sigma^2_0(k)), interleaved per height, and
//     A s = s - J(Lambda(T s)),   b = J t + c,
// with J including the factors 1-eps and W2 (Eq. 13-14).  One apply is
// Algorithm 1 itself:
//   k_sig_source   the source functions of every height and direction from
//                  the (right-preconditioned) input, Eq. (7)-(8);
//   the formal solver of the I-form path (k_formal, zero inflow) writes the
//                  radiation field of every ray into a scratch vector,
//                  Eq. (9)-(10);
//   k_sig_moments  J00 and J20 of that field per height, Eq. (11)-(12), and
//                  the output sigma - (xi J00, xi W2 J20).
// Right preconditioners act on the pair of one height: Jacobi scales by the
// inverse diagonal of A, local Lambda applies the inverse 2x2 block
// M_k = Id - J_k Lambda*_k T_k.
#include "rt_device.cuh"

namespace rt {

namespace {

constexpr int kSigThreads = 256;

// z_k = M^-1 v_k for the mode's right preconditioner
__device__ __forceinline__ void precond_pair(int mode, const double* __restrict__ v, const double* __restrict__ dinv,
                                             const double* __restrict__ Minv, int k, double& z0, double& z1) {
  const double v0 = v[2 * k], v1 = v[2 * k + 1];
  if (mode == KM_JACOBI) {
    z0 = v0 * dinv[2 * k];
    z1 = v1 * dinv[2 * k + 1];
  } else if (mode == KM_LOCAL_LAMBDA) {
    const double* M = Minv + 4 * k;
    z0 = M[0] * v0 + M[1] * v1;
    z1 = M[2] * v0 + M[3] * v1;
  } else {
    z0 = v0;
    z1 = v1;
  }
}

// S[s][k][m]: S_I = z0 + T201_m z1, S_Q = T202_m z1; KM_RHS: S = 0
template <int MODE>
__global__ void k_sig_source(const double* __restrict__ v, const double* __restrict__ dinv,
                             const double* __restrict__ Minv, const double* __restrict__ t201,
                             const double* __restrict__ t202, int Ns, int Nmu, double* __restrict__ S,
                             const int* kstop, int step) {
  if (kstop && step >= *kstop) return;
  const int64_t n = (int64_t)Ns * Nmu;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(i / Nmu), m = (int)(i % Nmu);
    if (MODE == KM_RHS) {
      S[i] = 0.0;
      S[n + i] = 0.0;
    } else {
      double z0, z1;
      precond_pair(MODE, v, dinv, Minv, k, z0, z1);
      S[i] = z0 + t201[m] * z1;
      S[n + i] = t202[m] * z1;
    }
  }
}

// one block per height: J00 = sum_r w_r I, J20 = sum_r w_r (T201_m I + T202_m Q)
// (w_r = hat-w_m hat-w_p), summed in a fixed order; then
//   apply: y_k = z_k - (xi J00, xi W2 J20);  KM_RHS: y_k = (xi J00 + eps B_k, xi W2 J20)
template <int MODE>
__global__ void __launch_bounds__(kSigThreads) k_sig_moments(
    const double* __restrict__ I, const double* __restrict__ v, const double* __restrict__ dinv,
    const double* __restrict__ Minv, const double* __restrict__ wray, const double* __restrict__ t201,
    const double* __restrict__ t202, const double* __restrict__ B, int Ns, int Nmu, int Nnu, double xi, double xiW2,
    double eps, double* __restrict__ y, const int* kstop, int step) {
  if (kstop && step >= *kstop) return;
  const int k = blockIdx.x;
  const int64_t nray = (int64_t)Nmu * Nnu;
  const double* __restrict__ Ik = I + (int64_t)k * nray;
  const double* __restrict__ Qk = I + ((int64_t)Ns + k) * nray;
  double a0 = 0.0, a2 = 0.0;
  for (int64_t r = threadIdx.x; r < nray; r += blockDim.x) {
    const int m = (int)(r / Nnu);
    const double wi = wray[r] * Ik[r];
    a0 += wi;
    a2 += t201[m] * wi + t202[m] * (wray[r] * Qk[r]);
  }
  __shared__ double red[2][kSigThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  a0 = warp_sum(a0);
  a2 = warp_sum(a2);
  if (lane == 0) {
    red[0][warp] = a0;
    red[1][warp] = a2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double j00 = 0.0, j20 = 0.0;
    for (int w = 0; w < kSigThreads / 32; ++w) {
      j00 += red[0][w];
      j20 += red[1][w];
    }
    const double s00 = xi * j00, s20 = xiW2 * j20;
    if (MODE == KM_RHS) {
      y[2 * k] = s00 + eps * B[k];
      y[2 * k + 1] = s20;
    } else {
      double z0, z1;
      precond_pair(MODE, v, dinv, Minv, k, z0, z1);
      y[2 * k] = z0 - s00;
      y[2 * k + 1] = z1 - s20;
    }
  }
}

// the paper's initial guess (Sect. 4.2): sigma^0_0 = 1, sigma^2_0 = 0 at every
// height, interleaved per height as the sigma-form vectors are
__global__ void k_sig_unit(int n, double* __restrict__ x) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] = (i & 1) ? 0.0 : 1.0;
}

// Jacobi diagonal of Eq. (18) (the diagonals of the blocks M_k), or its inverse
__global__ void k_sig_jacobi(const double* __restrict__ Mdiag, int n, int inverse, double* __restrict__ d) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    d[i] = inverse ? 1.0 / Mdiag[i] : Mdiag[i];
}

// z_k = M_k^-1 v_k
__global__ void k_sig_block(const double* __restrict__ v, const double* __restrict__ Minv, int Ns,
                            double* __restrict__ z, const int* kstop, int step) {
  if (kstop && step >= *kstop) return;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < Ns; k += gridDim.x * blockDim.x) {
    double z0, z1;
    precond_pair(KM_LOCAL_LAMBDA, v, nullptr, Minv, k, z0, z1);
    z[2 * k] = z0;
    z[2 * k + 1] = z1;
  }
}

// ------------------------------------------- SOR and SSOR (Sect. 2.3)
// The sigma-form matrix is small (n = 2*Ns), so the paper's SOR and SSOR
// preconditioners are formed densely from the assembled A = D + L + U and
// applied as one matrix-vector product (the paper precomputes the action of
// P^-1, Sect. 4.2).  Readings: the upper SOR variant P = D/omega + U, and
// SSOR P = omega/(2-omega) (D/omega + U) D^-1 (D/omega + L).

// e = unit vector j
__global__ void k_unit(double* __restrict__ e, int n, int j) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) e[i] = i == j ? 1.0 : 0.0;
}

// row-major A from column-major C (C[j*n + i] = A_ij)
__global__ void k_transpose(const double* __restrict__ C, int n, double* __restrict__ A) {
  const int64_t nn = (int64_t)n * n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nn; t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / n), j = (int)(t % n);
    A[t] = C[(int64_t)j * n + i];
  }
}

// X = (D/omega + U)^-1 (UPPER) or (D/omega + L)^-1, row-major: column j
// by back (forward) substitution in one thread; the threads of a warp read
// the same row of A and consecutive entries of a row of X
template <bool UPPER>
__global__ void k_tri_inverse(const double* __restrict__ A, int n, double omega, double* __restrict__ X) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  for (int s = 0; s < n; ++s) {
    const int i = UPPER ? n - 1 - s : s;
    double x = 0.0;
    if (UPPER ? i <= j : i >= j) {
      double r = i == j ? 1.0 : 0.0;
      if (UPPER)
        for (int k = i + 1; k <= j; ++k) r = fma(-A[(int64_t)i * n + k], X[(int64_t)k * n + j], r);
      else
        for (int k = j; k < i; ++k) r = fma(-A[(int64_t)i * n + k], X[(int64_t)k * n + j], r);
      x = r * omega / A[(int64_t)i * n + i];
    }
    X[(int64_t)i * n + j] = x;
  }
}

// M = c * Li * diag(A) * Ui with Li lower and Ui upper triangular (SSOR)
__global__ void k_ssor_product(const double* __restrict__ Li, const double* __restrict__ Ui,
                               const double* __restrict__ A, int n, double c, double* __restrict__ M) {
  const int64_t nn = (int64_t)n * n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nn; t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / n), j = (int)(t % n);
    const int kmax = i < j ? i : j;
    double s = 0.0;
    for (int k = 0; k <= kmax; ++k) s = fma(Li[(int64_t)i * n + k] * A[(int64_t)k * n + k], Ui[(int64_t)k * n + j], s);
    M[t] = c * s;
  }
}

// z = M v (row-major n x n), one warp per row
__global__ void k_gemv(const double* __restrict__ M, const double* __restrict__ v, int n, double* __restrict__ z,
                       const int* kstop, int step) {
  if (kstop && step >= *kstop) return;
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
    const double* __restrict__ row = M + (int64_t)i * n;
    double s = 0.0;
    for (int j = lane; j < n; j += 32) s = fma(row[j], v[j], s);
    s = warp_sum(s);
    if (lane == 0) z[i] = s;
  }
}

inline int blocks_for(int64_t n, int threads, int cap) {
  int64_t g = (n + threads - 1) / threads;
  return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

template <int MODE>
void launch_sigma(Problem* P, const double* v, double* y, cudaStream_t st, const int* kstop, int step) {
  const int Ns = P->Ns, Nmu = P->Nmu;
  k_sig_source<MODE><<<blocks_for((int64_t)Ns * Nmu, 256, 4 * P->num_sms), 256, 0, st>>>(
      v, P->dinv, P->Minv, P->t201d, P->t202d, Ns, Nmu, P->S, kstop, step); RT_COUNT(1);
  formal64_lambda(P, P->S, P->Ibuf, MODE == KM_RHS ? P->B[Ns - 1] : 0.0, st, kstop, step);
  k_sig_moments<MODE><<<Ns, kSigThreads, 0, st>>>(P->Ibuf, v, P->dinv, P->Minv, P->wray, P->t201d, P->t202d, P->Bd,
                                                   Ns, Nmu, P->Nnu, P->xi, P->xi * P->W2, P->eps, y, kstop, step);
  RT_COUNT(1);
}

}  // namespace

rt_status op_dense_precond_build(Problem* P, int kind, double omega, cudaStream_t st) {
  if (P->form != RT_FORM_SIGMA) {
    set_error("SOR and SSOR need the sigma-form (RT_FORM_SIGMA)");
    return RT_EINVAL;
  }
  const int n = (int)P->Nop;
  if (n > kMaxDenseN) {
    set_error("SOR and SSOR: the sigma-form system has %d > %d unknowns", n, kMaxDenseN);
    return RT_EINVAL;
  }
  if (!(omega > 0.0 && omega < 2.0)) {
    set_error("omega must be in (0, 2)");
    return RT_EINVAL;
  }
  const size_t nn = (size_t)n * n;
  // each buffer is allocated once; a failed allocation leaves the others for
  // the next call, and A is assembled only once all of them exist
  if (!P->Asig) RT_TRY_CUDA(dev_alloc(P, (void**)&P->Asig, nn * sizeof(double)));
  if (!P->Mpre) RT_TRY_CUDA(dev_alloc(P, (void**)&P->Mpre, nn * sizeof(double)));
  if (!P->Mtri) RT_TRY_CUDA(dev_alloc(P, (void**)&P->Mtri, nn * sizeof(double)));
  if (!P->Mscr) RT_TRY_CUDA(dev_alloc(P, (void**)&P->Mscr, 2 * (size_t)n * sizeof(double)));
  if (!P->asig_ready) {
    // the columns A e_j (one sigma-form apply each) into Mtri, then row-major
    for (int j = 0; j < n; ++j) {
      k_unit<<<blocks_for(n, 256, 64), 256, 0, st>>>(P->Mscr, n, j); RT_COUNT(1);
      RT_TRY(op_apply_sigma(P, P->Mscr, P->Mtri + (size_t)j * n, AM_PLAIN, st, nullptr, 0));
    }
    k_transpose<<<blocks_for((int64_t)nn, 256, 8 * P->num_sms), 256, 0, st>>>(P->Mtri, n, P->Asig); RT_COUNT(1);
    RT_TRY_CUDA(cudaGetLastError());
    P->asig_ready = 1;
    P->mpre_kind = 0;
  }
  const int base = (kind == RT_PREC_SOR || kind == RT_PREC_SOR_LEFT) ? RT_PREC_SOR : RT_PREC_SSOR;
  if (P->mpre_kind == base && P->mpre_omega == omega) return RT_OK;
  P->mpre_kind = 0;   // Mpre is rewritten below; tagged again once complete
  const int tb = 128, gb = (n + tb - 1) / tb;
  if (base == RT_PREC_SOR) {
    k_tri_inverse<true><<<gb, tb, 0, st>>>(P->Asig, n, omega, P->Mpre); RT_COUNT(1);
  } else {
    // P^-1 = (2-omega)/omega (D/omega + L)^-1 D (D/omega + U)^-1
    double* Li = nullptr;
    RT_TRY_CUDA(dev_alloc(P, (void**)&Li, nn * sizeof(double)));
    k_tri_inverse<true><<<gb, tb, 0, st>>>(P->Asig, n, omega, P->Mtri); RT_COUNT(1);
    k_tri_inverse<false><<<gb, tb, 0, st>>>(P->Asig, n, omega, Li); RT_COUNT(1);
    k_ssor_product<<<blocks_for((int64_t)nn, 256, 16 * P->num_sms), 256, 0, st>>>(Li, P->Mtri, P->Asig, n,
                                                                                (2.0 - omega) / omega, P->Mpre);
    RT_COUNT(1);
    const cudaError_t e = cudaStreamSynchronize(st);   // Li is freed on return
    dev_free(P, Li);
    RT_TRY_CUDA(e);
  }
  RT_TRY_CUDA(cudaGetLastError());
  P->mpre_kind = base;
  P->mpre_omega = omega;
  return RT_OK;
}

rt_status op_dense_precond_apply(Problem* P, const double* v, double* z, cudaStream_t st, const int* kstop,
                                 int step) {
  const int n = (int)P->Nop;
  k_gemv<<<blocks_for((int64_t)n * 32, 256, 8 * P->num_sms), 256, 0, st>>>(P->Mpre, v, n, z, kstop, step);
  RT_COUNT(1);
  RT_TRY_CUDA(cudaGetLastError());
  return RT_OK;
}

rt_status op_apply_sigma(Problem* P, const double* v, double* y, int mode, cudaStream_t st, const int* kstop,
                         int step) {
  switch (mode) {
    case AM_PLAIN:
      launch_sigma<KM_PLAIN>(P, v, y, st, kstop, step);
      break;
    case AM_JACOBI:
      launch_sigma<KM_JACOBI>(P, v, y, st, kstop, step);
      break;
    case AM_LOCAL_LAMBDA:
      launch_sigma<KM_LOCAL_LAMBDA>(P, v, y, st, kstop, step);
      break;
    default:
      set_error("bad apply mode");
      return RT_EINVAL;
  }
  RT_TRY_CUDA(cudaGetLastError());
  return RT_OK;
}

rt_status op_rhs_sigma(Problem* P, double* b, cudaStream_t st) {
  launch_sigma<KM_RHS>(P, nullptr, b, st, nullptr, 0);
  RT_TRY_CUDA(cudaGetLastError());
  return RT_OK;
}

rt_status op_x0_paper_sigma(Problem* P, double* x, cudaStream_t st) {
  k_sig_unit<<<blocks_for(2 * (int64_t)P->Ns, 256, 4 * P->num_sms), 256, 0, st>>>(2 * P->Ns, x);
  RT_COUNT(1);
  RT_TRY_CUDA(cudaGetLastError());
  return RT_OK;
}

rt_status op_jacobi_sigma(Problem* P, double* d, int inverse, cudaStream_t st) {
  k_sig_jacobi<<<blocks_for(2 * (int64_t)P->Ns, 256, 4 * P->num_sms), 256, 0, st>>>(P->Mdiag, 2 * P->Ns, inverse, d);
  RT_COUNT(1);
  RT_TRY_CUDA(cudaGetLastError());
  return RT_OK;
}

rt_status op_precond_sigma(Problem* P, const double* v, double* z, cudaStream_t st, const int* kstop, int step) {
  k_sig_block<<<blocks_for(P->Ns, 256, 4 * P->num_sms), 256, 0, st>>>(v, P->Minv, P->Ns, z, kstop, step);
  RT_COUNT(1);
  RT_TRY_CUDA(cudaGetLastError());
  return RT_OK;
}

}  // namespace rt

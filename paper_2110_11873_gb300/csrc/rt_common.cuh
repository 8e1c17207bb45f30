// Internal declarations of the GB300 transfer-operator library.
//
// Device layout of the I-form vector (Eq. 19): x[s][k][m][p], p fastest; the
// Nmu*Nnu rays of one height are contiguous.  Directions are stored mu
// ascending, so m < Nh (Nh = Nmu/2) are the downward rays (mu < 0, entering at
// the top, k = 0) and m >= Nh the upward rays (entering at the bottom).  The
// formal-solver coefficients depend on |mu| only, indexed mm = |m - Nh + 1/2| - 1/2:
//   mm = Nh-1-m (m < Nh),  mm = m-Nh (m >= Nh).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/rt_krylov.h"

namespace rt {

// NVTX range over the enclosing scope: named ranges for every entry point,
// solve phase and kernel launch, visible to profilers (no cost without one).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
#define RT_NVTX_CAT2(a, b) a##b
#define RT_NVTX_CAT(a, b) RT_NVTX_CAT2(a, b)
#define RT_NVTX(name) ::rt::NvtxRange RT_NVTX_CAT(rt_nvtx_, __LINE__)(name)

void set_error(const char* fmt, ...);
void clear_error();

// launch accounting for rt_launch_count(): launches issued while a graph is
// being captured are not counted; a graph launch counts its kernel nodes
extern thread_local int g_capturing;
void count_launches(long long n);
#define RT_COUNT(n)                                  \
  do {                                               \
    if (!::rt::g_capturing) ::rt::count_launches(n); \
  } while (0)

#define RT_TRY_CUDA(call)                                                                   \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) {                                                                \
      ::rt::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,     \
                      __LINE__);                                                            \
      return e_ == cudaErrorMemoryAllocation ? RT_ENOMEM : RT_ECUDA;                        \
    }                                                                                       \
  } while (0)

#define RT_TRY(expr)                 \
  do {                               \
    rt_status s_ = (expr);           \
    if (s_ != RT_OK) return s_;      \
  } while (0)

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// ---------------------------------------------------------------- kernels
// number of SMs on the device (152 on GB300), queried once per problem
constexpr int kBlockVec = 512;          // threads per block of the vector kernels
constexpr int kMaxPartials = 2048;      // upper bound on reduction partials per column
constexpr int kMaxRestart = 160;         // longest GMRES cycle (the paper runs GMRES unrestarted, up to 134 steps)
constexpr int kGramB = 4;                // basis vectors per block pass of the GMRES Arnoldi step

// device-side state of a GMRES cycle (lives in device memory).  The scalars
// come first: the host reads only that header (kGmresHeader bytes) after a
// cycle; the arrays are written before they are read within a cycle.
struct GmresDev {
  double bnorm, tol, rnorm, rel;   // ||b||, rtol, last true residual norm, rnorm/bnorm
  double vscale;                   // 1 / ||w|| of the current Arnoldi step (batched solver)
  double est;                      // |g_{j+1}| / ||b|| of the last Arnoldi step (Givens rotations)
  int kstop;                       // steps this cycle may take (set at cycle start)
  int kdone;                       // steps completed this cycle
  int iters;                       // Arnoldi steps over all cycles
  int maxit;
  int breakdown;
  int hist_len;
  double H[(kMaxRestart + 1) * kMaxRestart];  // column-major (m+1) x m, rotated in place
  double cs[kMaxRestart], sn[kMaxRestart];
  double g[kMaxRestart + 1];
  double y[kMaxRestart];
  double gram[(kMaxRestart + 1) * kGramB];   // gram[i*kGramB + d] = <v_i, v_{i-d}>, d = 1..kGramB-1
};
constexpr size_t kGmresHeader = offsetof(GmresDev, H);

// Programmatic dependent launch.  A kernel launched by launch_pdl may start
// while the stream's previous kernel drains; before it touches anything that
// kernel wrote it waits in pdl_wait (griddepcontrol.wait: the previous grid
// has completed and its writes are visible).  pdl_launch_dependents lets the
// next such kernel start; a kernel that never calls it releases its
// dependents as its CTAs exit.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// launch as a programmatic dependent of the stream's previous kernel
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), int grid, int block, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// sum of G partials in a fixed order (lane-strided, then a fixed shuffle
// tree); every lane of the calling warp gets the result
__device__ __forceinline__ double partials_sum_warp(const double* __restrict__ part, int G) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int i = lane; i < G; i += 32) s += part[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// Givens rotations on column j of the Hessenberg matrix and the residual
// estimate of GMRES (one thread)
__device__ inline void givens_step(GmresDev* gm, int m, int j, double* hist, int hist_cap) {
  double* Hc = gm->H + j * (m + 1);
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
  if (hist && gm->hist_len < hist_cap) hist[gm->hist_len++] = est;
  if (!(est >= gm->tol) || gm->iters >= gm->maxit || b == 0.0) gm->kstop = j + 1;
}

// End of Arnoldi step j from the last block pass's partials (Gp per set; set
// 0: ||w||^2, set 1+k: <w, v_{i0+k}>, k < ng): h_{j+1,j} = ||w|| to
// hcol[j+1], the Gram row j+1 (<v_{j+1}, v_{j+1-d}>, d = ng - k), and with
// gm set the Givens rotations of column j.  One CTA of at least 32*(1+ng)
// threads; thread 0 does the scalar work.
__device__ inline void arnoldi_fold(const double* __restrict__ part, int Gp, int ng, double* __restrict__ hcol,
                                    double* __restrict__ gram, GmresDev* gm, int m, int j, double* hist,
                                    int hist_cap) {
  __shared__ double sets[kGramB];
  const int warp = threadIdx.x >> 5;
  if (warp <= ng) {
    const double s = partials_sum_warp(part + (size_t)warp * Gp, Gp);
    if ((threadIdx.x & 31) == 0) sets[warp] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double hn = sqrt(sets[0]);
    const double inv = hn > 0.0 ? 1.0 / hn : 0.0;
    hcol[j + 1] = hn;
    for (int d = 1; d <= ng; ++d) gram[(j + 1) * kGramB + d] = sets[1 + ng - d] * inv;
    if (gm) givens_step(gm, m, j, hist, hist_cap);
  }
}

// 1 / ||w|| from set 0 of the same partials, in the same summation order as
// arnoldi_fold (0 for a zero norm), broadcast to the CTA
__device__ inline double arnoldi_inv_norm(const double* __restrict__ part, int Gp) {
  __shared__ double inv_s;
  if (threadIdx.x < 32) {
    const double s = partials_sum_warp(part, Gp);
    if (threadIdx.x == 0) {
      const double h = sqrt(s);
      inv_s = h > 0.0 ? 1.0 / h : 0.0;
    }
  }
  __syncthreads();
  const double inv = inv_s;
  __syncthreads();
  return inv;
}

// transposing warp reduction of four FP64 values (6 additions a lane instead
// of 20): lane l gets the warp sum of s[2*((l>>4)&1) + ((l>>3)&1)], so lanes
// 0, 8, 16 and 24 hold the sums of s[0], s[1], s[2] and s[3]; fixed order
__device__ __forceinline__ double warp_sum4(const double* s) {
  const int lane = threadIdx.x & 31;
  const bool h16 = lane & 16, h8 = lane & 8;
  const double r0 = (h16 ? s[2] : s[0]) + __shfl_xor_sync(0xffffffffu, h16 ? s[0] : s[2], 16);
  const double r1 = (h16 ? s[3] : s[1]) + __shfl_xor_sync(0xffffffffu, h16 ? s[1] : s[3], 16);
  double t = (h8 ? r1 : r0) + __shfl_xor_sync(0xffffffffu, h8 ? r0 : r1, 8);
  t += __shfl_xor_sync(0xffffffffu, t, 4);
  t += __shfl_xor_sync(0xffffffffu, t, 2);
  t += __shfl_xor_sync(0xffffffffu, t, 1);
  return t;
}

// device-side scalars of BiCGSTAB / CGS
struct BicgDev {
  double rho, rho_old, alpha, omega, beta;
  double bnorm, tol, rel;
  int done;        // 1 converged, 2 breakdown, 3 numeric
  int iters;
  int maxit;
  int half;        // BiCGSTAB converged at the half step
};

// Column of the FP64 step-coefficient tables for ray r = m*Nnu + p.  Without
// a downwind term the coefficients of a step depend on |mu| only, so the
// tables hold one column per (|mu|, p) that both directions share (shared =
// 1, nray/2 columns): m < Nh (mu < 0) reads column (Nh-1-m)*Nnu + p, m >= Nh
// column (m-Nh)*Nnu + p.  DELO-parabolic's coefficients include the downwind
// interval, which differs between the directions: one column per ray.
__host__ __device__ __forceinline__ int64_t coef_col(int64_t r, int Nh, int Nnu, int shared) {
  if (!shared) return r;
  const int m = (int)(r / Nnu);
  const int64_t p = r - (int64_t)m * Nnu;
  return (int64_t)(m < Nh ? Nh - 1 - m : m - Nh) * Nnu + p;
}

// Device memory source of a problem: NULL means cudaMalloc/cudaFree; the
// batch server passes its arena; rt_problem_create_with_allocator the
// caller's hook.
struct DevAllocator {
  virtual ~DevAllocator() {}
  virtual cudaError_t alloc(void** p, size_t bytes) = 0;
  virtual void release(void* p) = 0;
};

// A caller-provided rt_allocator behind the DevAllocator interface: every
// request goes to the hook with the stream the object was made with; the
// sizes are remembered for the matching release.  Blocks must be 256-byte
// aligned (a misaligned one is handed back and the request fails).
DevAllocator* make_hook_allocator(const rt_allocator* hook, cudaStream_t st);

struct Problem {
  DevAllocator* alloc = nullptr;     // NULL: cudaMalloc / cudaFree
  DevAllocator* own_alloc = nullptr; // the caller's allocator hook, owned (deleted at destroy)
  int in_arena = 0;                  // 1: an instance of the batch server, tables in its arena
  // sizes
  int Ns = 0, Nmu = 0, Nnu = 0, Nh = 0;
  int64_t nray = 0;   // Nmu*Nnu rays per Stokes parameter
  int64_t N = 0;      // 2*Ns*nray: length of the radiation field (the I-form unknown)
  int form = 0;       // RT_FORM_I or RT_FORM_SIGMA: the system the solvers and rt_apply work on
  int64_t Nop = 0;    // length of that system's vectors: N (I-form) or 2*Ns (sigma-form)
  int device = 0, num_sms = 0;
  // physics
  double eps = 0, xi = 0, W2 = 0, a = 0;
  int tau_kind = 0, mu_quad = 0, fs = 0, freq_norm = 0;
  // host grids
  std::vector<double> tau, B, mu, w_mu, x, phi, w_nu, phi_hat, t201, t202;
  // ray groups of the formal-solver kernel: 32 consecutive rays of one
  // direction sign; the nd = Nh*Nnu downward rays come first
  int64_t nd = 0;
  int ngroups = 0;
  int ntile64 = 1, ntile32 = 1;   // depth tiles per ray group (FP64 / FP32 kernels)
  // FP64 device tables
  int cshare = 0;          // 1: the FP64 tables hold one column per (|mu|, p), shared by both directions
  int64_t cstride = 0;     // columns of the FP64 tables: nray/2 (shared) or nray (DELO-parabolic)
  double* ce = nullptr;    // [(Ns-1)][cstride] step factor e of the interval (i, i+1), column coef_col(r)
  double* ca = nullptr;    // ... alpha (coefficient of the upwind S)
  double* cb = nullptr;    // ... beta  (coefficient of S at the new node)
  double* cg = nullptr;    // ... gamma (DELO-parabolic only: coefficient of S at the downwind node)
  double* Etile = nullptr; // [ntile64-1][nray] FP64 formal solver: slope of each depth tile's map
  // sigma-form SOR / SSOR: the assembled matrix A (row-major n x n, n = Nop),
  // the dense P^-1 (row-major), a triangular-inverse scratch and a vector
  double *Asig = nullptr, *Mpre = nullptr, *Mtri = nullptr, *Mscr = nullptr;
  int asig_ready = 0;        // Asig holds the assembled matrix
  int mpre_kind = 0;         // RT_PREC_SOR / RT_PREC_SSOR that Mpre holds (0: none)
  double mpre_omega = 0.0;
  double* Bmap = nullptr;  // [2*ngroups][ntile64-1][32] FP64 formal solver: offsets of the tile maps
  double* Kmap = nullptr;  // [ntile64-1][L+2][nray] weights of the map offsets in the node source values
  double* wray = nullptr;  // [3][nray] hat-w_m * hat-w_p, the same times T201_m, times T202_m
  double* wjac = nullptr;  // [3][Ns][nray] wray times the Jacobi inverse diagonal (I, I, Q), once a solver set it
  double* wI2 = nullptr;   // [Nnu] spectral weights hat-w_p
  double* wQ2 = nullptr;   // [Nmu] angular weights hat-w_m = w_m / 2
  double* t201d = nullptr; // [Nmu]
  double* t202d = nullptr; // [Nmu]
  double* Bd = nullptr;    // [Ns]
  double* Minv = nullptr;  // [Ns][4] inverse of the 2x2 local blocks M_k (row-major)
  double* Mdiag = nullptr; // [Ns][2] diagonal of M_k (the sigma-form Jacobi diagonal)
  double* Ibuf = nullptr;  // sigma-form only: [2][Ns][nray] radiation field of one apply
  double* S = nullptr;     // [2][Ns][Nmu] source-function scratch
  double* S2 = nullptr;    // second source-function scratch
  // FP32 device tables
  float* dtau32 = nullptr;  // [Ns-1] tau_{k+1} - tau_k
  float* r32 = nullptr;     // [nray] phi_hat_p / |mu_m|
  float* wray32 = nullptr;
  float* wI2f = nullptr;
  float* wQ2f = nullptr;
  float* t201f = nullptr;
  float* t202f = nullptr;
  float* S32 = nullptr;     // [2][Ns][Nmu]
  // solver workspace (allocated on first use)
  int ws_restart = 0;
  double* V = nullptr;        // (restart+1) vectors of N
  double* work = nullptr;     // 8 work vectors of N
  double* dinv = nullptr;     // N, Jacobi inverse diagonal
  float* work32 = nullptr;    // 2 vectors of N (FP32 operator)
  double* partials = nullptr; // 2 x kMaxPartials x 8
  double* bpart = nullptr;    // 3 x kGramB x kMaxPartials: block-pass partials (two ping-pong buffers, Gram)
  GmresDev* gm = nullptr;
  BicgDev* bc = nullptr;
  double* hist = nullptr;     // device history
  int hist_cap_dev = 0;
  int vec_grid = 0;           // blocks of the reduction kernels
  // fast FP32 apply (rt_tma.cu): usable for this problem, its tables, and
  // the device flag its bounded waits set when they give up
  int staged = 0;
  int ntile_st = 1;            // depth tiles per ray group of the staged formal solver
  int quad_gx = 1, quad_gy = 1, quad_hpc = 1;   // quadrature grid, heights per CTA
  int quadn_gy = 1, quadn_hpc = 1;             // the same for the fused-normalisation quadrature
  float* qw = nullptr;         // [3][nray] quadrature weights w0, w0*T201, w0*T202
  float4* stab = nullptr;      // [2][Ns + pad] node operands of the formal solver, march-indexed per
                               // direction: (sigma00, sigma20) of the node, then the constants of the
                               // interval a step into it crosses
  float* qpart = nullptr;      // [Ns][quad_gx][2] partial moments
  int* qcnt = nullptr;         // [quadrature grid rows] CTAs of a row done (the last one forms sigma)
  int* dev_err = nullptr;
  float* tile_dt = nullptr;    // [2][ntile_st] DELO-linear: the sum of dtau / ln 2 over each depth tile
  void* tma_cache = nullptr;   // host: recently encoded tensor maps of the FP32 apply (rt_tma.cu)
  int inject_wait_fail = 0;    // standalone FP32 applies still to run with one tensor-copy wait forced to
                               // give up (failure injection, rt_problem_inject_wait_timeout)
};

// operator entry points used by the solvers (all enqueue on `st`)
enum ApplyMode { AM_PLAIN = 0, AM_JACOBI = 1, AM_LOCAL_LAMBDA = 2 };
// kstop/step: inside a captured GMRES cycle the kernels of Arnoldi step
// `step` return at once when step >= *kstop (NULL: always run)
// GMRES, FP64 I-form: the normalisation that ends Arnoldi step jprev done by
// the apply of step jprev + 1.  Its quadrature kernel reads u (the last block
// pass's w), writes x = u / ||u|| as it goes, and one CTA folds h and the
// Gram row and applies the Givens rotations of column jprev (arnoldi_fold).
struct NormIn {
  const double* u;
  const double* part;   // the last pass's partials: set 0 ||u||^2, sets 1..ng the Gram dots
  int Gp, ng;
  double* hcol;         // column jprev of the Hessenberg matrix
  double* gram;
  GmresDev* gm;
  int m, jprev;
  double* hist;
  int hist_cap;
  const int* kstop;     // the kernel runs while jprev < *kstop
};
rt_status op_apply64(Problem* P, const double* x, double* y, int mode, cudaStream_t st,
                     const int* kstop = nullptr, int step = 0, const NormIn* nin = nullptr);
rt_status op_apply32(Problem* P, const float* x, float* y, int mode, cudaStream_t st);
rt_status op_apply32_f64io(Problem* P, const double* x, double* y, int mode, cudaStream_t st,
                           const int* kstop = nullptr, int step = 0, const NormIn* nin = nullptr);
rt_status op_precond_ll(Problem* P, const double* v, double* z, cudaStream_t st, const int* kstop = nullptr,
                        int step = 0);
rt_status op_jacobi_inv(Problem* P, double* dinv, cudaStream_t st);
// the Jacobi-mode quadrature weights from P->dinv (I-form; the apply in
// Jacobi mode uses them once they exist)
rt_status op_jacobi_weights(Problem* P, cudaStream_t st);
rt_status op_rhs(Problem* P, double* b, cudaStream_t st);
// the paper's initial guess (Sect. 4.2) in the problem's form: sigma =
// [1, 0, 1, 0, ...], or for the I-form Lambda(T sigma) + t
rt_status op_x0_paper(Problem* P, double* x, cudaStream_t st);
void release_graphs(Problem* P);
// the formal solver alone (Eq. 9-10): I = Lambda S with the given inflow at
// the bottom for Stokes I (zero elsewhere), FP64, written to I_out [2][Ns][nray]
void formal64_lambda(Problem* P, const double* S, double* I_out, double inflow_bottom, cudaStream_t st,
                     const int* kstop = nullptr, int step = 0);
// sigma-form operator and its companions (rt_sigma.cu); vectors of 2*Ns
rt_status op_apply_sigma(Problem* P, const double* v, double* y, int mode, cudaStream_t st,
                         const int* kstop = nullptr, int step = 0);
rt_status op_rhs_sigma(Problem* P, double* b, cudaStream_t st);
rt_status op_x0_paper_sigma(Problem* P, double* x, cudaStream_t st);   // [1, 0, 1, 0, ...]
rt_status op_jacobi_sigma(Problem* P, double* d, int inverse, cudaStream_t st);
// sigma-form SOR / SSOR (kind RT_PREC_SOR or RT_PREC_SSOR, with or without
// _LEFT): assemble A on first use, form P^-1 for (kind, omega) in Mpre
rt_status op_dense_precond_build(Problem* P, int kind, double omega, cudaStream_t st);
// z = P^-1 v with the Mpre of the last build (one GEMV)
rt_status op_dense_precond_apply(Problem* P, const double* v, double* z, cudaStream_t st, const int* kstop = nullptr,
                                 int step = 0);
constexpr int kMaxDenseN = 8192;   // largest sigma-form system with a dense SOR / SSOR inverse
rt_status op_precond_sigma(Problem* P, const double* v, double* z, cudaStream_t st, const int* kstop = nullptr,
                           int step = 0);
// fast FP32 apply (rt_tma.cu)
rt_status staged_setup(Problem* P, cudaStream_t st);
void staged_release(Problem* P);   // host state of the fast FP32 apply
bool staged_apply32(Problem* P, const void* x, void* y, bool f64io, int mode, cudaStream_t st, const int* kstop,
                    int step, rt_status* status, const NormIn* nin = nullptr);
// whether staged_apply32 takes FP64 vectors x (and a normalisation input u)
// in this apply mode
bool staged_f64io_ok(const Problem* P, int mode, const void* x, const void* u);
// RT_ETIMEOUT (and clears the flag) when a bounded device wait gave up
rt_status check_device_flag(Problem* P, cudaStream_t st);
rt_status setup_device_tables(Problem* P, cudaStream_t st);
void free_device(Problem* P);
rt_status validate_desc(const rt_problem_desc* d);
void host_grids(const rt_problem_desc* d, Problem& P);
cudaError_t dev_alloc(Problem* P, void** p, size_t bytes);
// Debug aid: with RT_POISON=1 in the environment every new workspace (of a
// problem, of the batch server, and every block the server's arena hands
// out) is filled with 0xFF bytes -- NaN in FP64 and FP32, -1 in integers --
// before it is returned, so a kernel that reads memory nothing has written
// yet produces NaN instead of a plausible stale value.  Off by default; not
// inside a stream capture.
cudaError_t poison_fill(void* p, size_t bytes);
void dev_free(Problem* P, void* p);

}  // namespace rt

struct rt_problem {
  rt::Problem P;
};

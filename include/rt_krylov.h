/*
 * rt_krylov.h -- C ABI of the GB300 (sm_103a) matrix-free transfer operator and
 * Krylov solvers for the 1D two-level-atom CRD polarized transfer problem of
 * Benedusi, Janett, Belluzzi & Krause (2021), "Numerical solutions to linear
 * transfer problems of polarized radiation II" (Sect. 3-4).
 *
 * Unknown: the I-form vector of Eq. (19), the Stokes I and Q radiation field
 * at every height z_k, direction mu_m and frequency nu_p:
 *
 *     x[s][k][m][p],  s = 0 (I), 1 (Q);  k = 0..Ns-1 (top, smallest tau, to
 *     bottom);  m = 0..Nmu-1 (mu ascending: the Nmu/2 downward directions
 *     first);  p = 0..Nnu-1 (reduced frequency ascending);
 *     flat index ((s*Ns + k)*Nmu + m)*Nnu + p,  length N = 2*Ns*Nmu*Nnu.
 *
 * Operator (Eq. 19, Algorithm 1 transposed to the I-form):
 *     A x = x - Lambda(T(J x)),
 *   J: sigma00_k = xi * J00_k, sigma20_k = xi * W2 * J20_k  (Eq. 11-14, xi = 1-eps)
 *   T: S_I(k,m) = sigma00_k + T201(mu_m) sigma20_k, S_Q(k,m) = T202(mu_m) sigma20_k (Eq. 7-8)
 *   Lambda: formal solution of Eq. (9)-(10) along every (m,p) ray with zero inflow.
 * Right-hand side (Eq. 19): b = Lambda T c + t with c = [eps B_k, 0] and the
 * boundary conditions after Eq. (10) (I = B(tau_Ns), Q = 0 entering at the
 * bottom for mu > 0; nothing entering at the top).
 *
 * Memory: every vector argument named *_dev is caller-owned device memory on
 * the device that was current at rt_problem_create; the library never frees
 * it and keeps no pointer to it after the call returns.  Host arrays in
 * rt_problem_desc are copied by rt_problem_create.  The problem owns its
 * device workspaces (coefficient tables, Krylov basis) until
 * rt_problem_destroy.  `stream` is a cudaStream_t (NULL = legacy default
 * stream); all device work of a call is ordered on it.  Calls on one problem
 * must not overlap in time (one host thread at a time, one stream at a time).
 *
 * Errors: every entry point returns an rt_status and never throws;
 * rt_last_error() gives a thread-local message for the last failure.
 */
#ifndef RT_KRYLOV_H
#define RT_KRYLOV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RT_OK = 0,
  RT_EINVAL = 1,       /* invalid argument; nothing was launched */
  RT_ENOMEM = 2,       /* device allocation failed */
  RT_ECUDA = 3,        /* a CUDA runtime call failed; see rt_last_error() */
  RT_ENOTCONV = 4,     /* maxit reached: x_dev holds the last iterate */
  RT_EBREAKDOWN = 5,   /* Krylov breakdown (zero denominator); x_dev holds the last iterate */
  RT_ENUMERIC = 6,     /* NaN or Inf met in a residual */
  RT_EPENDING = 7,     /* batch ticket not finished yet */
  RT_ETIMEOUT = 8,     /* a device-side bounded wait gave up */
  RT_ECANCELED = 9     /* batch request cancelled (rt_batch_cancel) or past its deadline */
} rt_status;

/* optical-depth convention (reading of Sect. 4.1): the tau grid is line-centre
   optical depth (path depth at frequency p scaled by H(a,x_p)/H(a,0)) or
   frequency-integrated optical depth (scaled by phi(x_p) = H(a,x_p)/sqrt(pi)) */
enum { RT_TAU_LINE_CENTER = 0, RT_TAU_FREQ_INTEGRATED = 1 };
/* angular quadrature: Gauss-Legendre per hemisphere (Nmu/2 nodes on [0,1] and
   their mirror) or Nmu Gauss-Legendre nodes on [-1,1] (Sect. 4.1) */
enum { RT_MU_GL_HALF = 0, RT_MU_GL_FULL = 1 };
/* formal solver (Sect. 4.1): DELO-linear, implicit Euler, trapezoidal, and
   DELO-parabolic (the exponential integrator with the source function
   interpolated by the parabola through the upwind, current and downwind
   nodes; the paper names the parabolic DELO methods without formulas).
   DELO-parabolic is FP64 only: rt_apply_f32, RT_PRECISION_FP32_REFINE and the
   batch server reject it.  RT_FS_DELOPAR names the same scheme: the paper
   lists DELOPAR and DELO-parabolic side by side, with no formulas for
   either, and here the propagation matrix is eta_I times the identity (no
   dichroism), so both are read as this one parabolic exponential
   integrator. */
enum {
  RT_FS_DELO_LINEAR = 0,
  RT_FS_IMPLICIT_EULER = 1,
  RT_FS_TRAPEZOIDAL = 2,
  RT_FS_DELO_PARABOLIC = 3,
  RT_FS_DELOPAR = RT_FS_DELO_PARABOLIC
};
/* linear system (Sect. 3.2):
   RT_FORM_I      Eq. (19): unknown I, N = 2*Ns*Nmu*Nnu values x[s][k][m][p],
                  A x = x - Lambda(T(J x)), b = Lambda T c + t;
   RT_FORM_SIGMA  Eq. (18): unknown sigma, N = 2*Ns values interleaved per
                  height (sigma^0_0(k), sigma^2_0(k)), A s = s - J(Lambda(T s))
                  with J including the factors 1-eps and W2, b = J t + c.
                  The sigma-form operator is FP64 in every precision; the
                  batch server takes I-form problems only. */
enum { RT_FORM_I = 0, RT_FORM_SIGMA = 1 };

typedef struct {
  int32_t Ns;              /* heights, >= 2 */
  int32_t Nmu;             /* directions, even, >= 2, <= 256 */
  int32_t Nnu;             /* frequencies, >= 2 */
  const double* tau;       /* host, Ns strictly increasing optical depths (required) */
  const double* B;         /* host, Ns Planck values, or NULL for B = 1 */
  const double* phi;       /* host, Nnu profile values phi(x_p) = H(a,x_p)/sqrt(pi), or
                              NULL to compute the Voigt profile internally (needs 0 < a <= 0.1);
                              for RT_TAU_LINE_CENTER, phi at x = 0 is taken as
                              phi_center (below) */
  double phi_center;       /* used only when phi != NULL and tau_kind is line-centre:
                              phi(0) = H(a,0)/sqrt(pi) */
  double x_min, x_max;     /* uniform reduced-frequency grid, x_min < x_max */
  double a;                /* Voigt damping (Sect. 3.1: 1e-3) */
  double eps;              /* thermalisation parameter, 0 < eps <= 1 (Eq. 13) */
  double W2;               /* polarizability factor on sigma^2_0 (Eq. 14: 1) */
  int32_t tau_kind;        /* RT_TAU_* */
  int32_t mu_quad;         /* RT_MU_* */
  int32_t formal_solver;   /* RT_FS_* */
  int32_t freq_norm;       /* 1: divide the trapezoidal spectral weights by their sum;
                              0: plain trapezoid (the paper's tables) */
  int32_t form;            /* RT_FORM_*: the linear system rt_apply, rt_rhs,
                              rt_jacobi_diag, rt_precond_local_lambda and the
                              solvers work on (0, the I-form, when unset) */
} rt_problem_desc;

typedef struct rt_problem rt_problem;

/* Build grids, profile and coefficient tables for one atmosphere (Sect. 3.2,
   4.1).  Device workspaces are allocated here.  RT_EINVAL for Ns < 2, odd or
   out-of-range Nmu, Nnu < 2, eps outside (0,1], a <= 0 (or a > 0.1 with
   phi == NULL), non-increasing tau, x_min >= x_max, unknown enums. */
rt_status rt_problem_create(const rt_problem_desc* desc, void* stream, rt_problem** out);
rt_status rt_problem_destroy(rt_problem* prob);

/* Device memory from the caller (the paper has no counterpart: this is how
   the library's workspaces can come from another allocator, such as
   PyTorch's caching allocator, which then accounts for them).
     alloc(ctx, bytes, stream)   returns `bytes` of device memory on the
                                 current device, aligned to 256 bytes or
                                 more, or NULL when it cannot;
     release(ctx, ptr, bytes, stream)  takes back a block alloc returned,
                                 with the size it was asked for.
   `stream` is the stream given to rt_problem_create_with_allocator (for a
   server: the server's internal stream); the library uses a block only on
   the streams of its own calls, which never overlap in time for one problem.
   Both functions are called from the thread making the library call, and for
   a server also from its worker thread; they must not call back into this
   library.  A request the library cannot satisfy fails with RT_ENOMEM. */
typedef struct {
  void* ctx;
  void* (*alloc)(void* ctx, size_t bytes, void* stream);
  void (*release)(void* ctx, void* ptr, size_t bytes, void* stream);
} rt_allocator;

/* rt_problem_create with every device workspace of the problem -- the
   tables built here, the Krylov basis, work vectors and GMRES state (taken
   at the first solve), the residual history -- requested from `allocator`
   instead of cudaMalloc.  The rt_allocator struct is copied; its functions
   and ctx must stay valid until rt_problem_destroy has returned, which
   synchronises the device and then releases every block.  allocator NULL
   behaves as rt_problem_create; RT_EINVAL when alloc or release is NULL. */
rt_status rt_problem_create_with_allocator(const rt_problem_desc* desc, const rt_allocator* allocator, void* stream,
                                           rt_problem** out);
/* Length N of the system's vectors: 2*Ns*Nmu*Nnu (RT_FORM_I) or 2*Ns
   (RT_FORM_SIGMA); -1 for NULL */
int64_t rt_problem_size(const rt_problem* prob);

/* Host copies of the discrete grids (any pointer may be NULL):
   mu[Nmu], w_mu[Nmu] (sum 2), x[Nnu], phi[Nnu], w_nu[Nnu] (spectral weights,
   sum 1 with freq_norm), phi_hat[Nnu] (optical-depth scale per frequency). */
rt_status rt_problem_grids(const rt_problem* prob, double* mu, double* w_mu, double* x,
                           double* phi, double* w_nu, double* phi_hat);

/* y = x - Lambda(T(J x))   (Eq. 19; Algorithm 1), or for RT_FORM_SIGMA
   y = s - J(Lambda(T s)) (Eq. 18; Algorithm 1 itself).  x_dev, y_dev: N
   doubles, distinct buffers.  FP64 throughout. */
rt_status rt_apply(rt_problem* prob, const double* x_dev, double* y_dev, void* stream);

/* Same operator with FP32 vectors and FP32 quadrature and formal solver
   (coefficients recomputed in FP32 with the small-Delta series).  When the
   layout allows (Nmu*Nnu and Nmu/2*Nnu multiples of 4, x_dev 16-byte
   aligned) the formal solver streams x through shared memory with tensor
   copies whose waits are bounded; a wait that gives up leaves y invalid and
   is reported by rt_problem_check.  Setting RT_NO_TMA=1 in the environment
   before rt_problem_create selects the register-ring kernel instead.  The two
   kernels agree to FP32 rounding accumulated along the rays, not bit for bit:
   they split the depth scan into different tiles, sum the quadrature in
   different orders and carry the recurrence in different variables. */
rt_status rt_apply_f32(rt_problem* prob, const float* x_dev, float* y_dev, void* stream);

/* Synchronises `stream` and reports RT_ETIMEOUT (then clears the condition)
   when a bounded device-side wait of this problem's kernels gave up since the
   last check; RT_OK otherwise.  The paper has no counterpart: it guards this
   library's asynchronous copies.  rt_solve_gmres performs the same check
   before it returns. */
rt_status rt_problem_check(rt_problem* prob, void* stream);

/* Which formal-solver kernel the FP32 applies of this problem use (no
   counterpart in the paper): 1 = shared-memory tensor-copy staging, 0 = the
   register-ring kernel, -1 for NULL.  Host only. */
int rt_problem_formal_kernel(const rt_problem* prob);

/* Failure injection for the bounded waits (no counterpart in the paper; it
   exercises this library's error path without a device fault): the next
   `count` calls of rt_apply_f32 on this problem that take the tensor-copy
   kernel treat the first wait of one warp as given up -- that warp flags the
   problem, waits (bounded) for its copies in flight and skips its depth
   tile, so y is invalid and the next rt_problem_check returns RT_ETIMEOUT.
   count = 0 disarms it.  RT_EINVAL for NULL or count < 0.  Host only. */
rt_status rt_problem_inject_wait_timeout(rt_problem* prob, int32_t count);

/* b = Lambda T c + t of Eq. (19): one formal solve with S_I = eps B, S_Q = 0
   and the boundary radiation; for RT_FORM_SIGMA b = J t + c of Eq. (18), t
   the boundary radiation transmitted with S = 0.  b_dev: N doubles. */
rt_status rt_rhs(rt_problem* prob, double* b_dev, void* stream);

/* Diagonal of Id - Lambda T J (Jacobi P = D, Sect. 2.3):
   D_I = 1 - xi beta* w_m w_p (1 + W2 T201^2), D_Q = 1 - xi W2 beta* w_m w_p T202^2,
   beta* the coefficient of S_k in the last formal-solver step ending at k.
   For RT_FORM_SIGMA the diagonal of Eq. (18): the diagonals of the per-height
   blocks M_k = Id - J_k Lambda*_k T_k.  d_dev: N doubles. */
rt_status rt_jacobi_diag(rt_problem* prob, double* d_dev, void* stream);

/* z = P^{-1} v for the local-Lambda preconditioner P = Id - Lambda* T J
   (Lambda* the diagonal of Lambda): P^{-1} v = v + Lambda* T M^{-1} J v with
   M_k = Id - J_k Lambda*_k T_k the 2x2 per-height block of the sigma-form
   (Eq. 18).  This is the sigma-form block-Jacobi preconditioner of Sect. 2.3
   carried to the I-form by the Woodbury identity.  For RT_FORM_SIGMA the
   block-Jacobi preconditioner itself: z_k = M_k^{-1} v_k per height.
   v_dev, z_dev: N doubles. */
rt_status rt_precond_local_lambda(rt_problem* prob, const double* v_dev, double* z_dev, void* stream);

/* z = P^-1 v for the sigma-form SOR (kind RT_PREC_SOR) or SSOR
   (RT_PREC_SSOR) preconditioner with relaxation omega, 0 < omega < 2: the
   operators the solvers use with those preconditioners (defined with the
   RT_PREC_* values below; Sect. 2.3).  The first call for a problem
   assembles A (2*Ns applies), a call with a new (kind, omega) forms P^-1
   (stream-ordered, synchronising once); each call then does one dense
   matrix-vector product.  v_dev, z_dev: 2*Ns doubles, distinct.
   RT_EINVAL for the I-form or more than 8192 unknowns. */
rt_status rt_precond_stationary(rt_problem* prob, int32_t kind, double omega, const double* v_dev, double* z_dev,
                                void* stream);

/* One Arnoldi orthogonalisation step by modified Gram-Schmidt (Sect. 2.1:
   the O(nN) nested loop of GMRES), on the problem's vector length N:
     for i = 0..j: h_i = <w, v_i>; w -= h_i v_i;   h_{j+1} = ||w||;  v_{j+1} = w / h_{j+1}
   V_dev: j+2 vectors of N doubles, contiguous (v_i at V_dev + i*N), v_0..v_j
   orthonormal; v_{j+1} is written.  w_dev: N doubles, overwritten.
   h_dev: j+2 doubles (device), receives h_0..h_{j+1}.  0 <= j < 160.
   Reductions are deterministic (fixed block partials, fixed summation order). */
rt_status rt_arnoldi_mgs(rt_problem* prob, double* V_dev, int32_t j, double* w_dev, double* h_dev, void* stream);

/* One Arnoldi step by block modified Gram-Schmidt, the orthogonalisation
   inside rt_solve_gmres (Sect. 2.1; the coefficients of rt_arnoldi_mgs in
   exact arithmetic).  The basis is taken in blocks of RT_GRAM_BLOCK vectors:
   with r_k = <w, v_k> formed before a block's updates, modified Gram-Schmidt
   gives h_k = r_k - sum_{l<k} h_l <v_l, v_k> (l, k in the block), so one pass
   over the data applies a whole block and forms the dots with the next one.
   The paper has no block form; it is a reformulation of its MGS loop with the
   same FP64 operations per element and a quarter of the passes.
   gram_dev: (j+2) x RT_GRAM_BLOCK doubles; row i holds <v_i, v_{i-d}> in
   column d = 1..RT_GRAM_BLOCK-1 (column 0 unused).  Rows 1..j are read (all
   zero for an exactly orthonormal basis), each only in the columns whose
   vectors share its block (d <= i mod RT_GRAM_BLOCK).  For the new vector,
   row j+1 gets exactly those columns, d = 1..(j+1) mod RT_GRAM_BLOCK; its
   other columns are left as they are.  V_dev, w_dev, h_dev and the limits
   as rt_arnoldi_mgs. */
#define RT_GRAM_BLOCK 4
rt_status rt_arnoldi_bmgs(rt_problem* prob, double* V_dev, int32_t j, double* w_dev, double* gram_dev,
                          double* h_dev, void* stream);

/* The same MGS Arnoldi step for callers that cannot allocate device memory
   (code running while a stream is captured into a CUDA graph, processes whose
   device memory belongs to another allocator that must account for every
   byte, service loops that cannot afford the device synchronisation an
   allocation may cause).  The paper has no counterpart: this is a
   deployment variant of rt_arnoldi_mgs.
   It needs no rt_problem: N is the vector length, V_dev holds j+2 vectors of
   N doubles (v_0..v_j orthonormal; v_{j+1} is written), w_dev is overwritten,
   h_dev receives j+2 doubles; all caller-owned device memory.
   It calls no cudaMalloc, cudaFree or allocating library routine.  Its only
   scratch, the per-block partial sums of the reductions, is a static device
   array of 2 x 1024 doubles (16 KB) inside the library, which every GPU that
   loads the library keeps until the process exits.  The first call on a
   device looks up that array's device address (cudaGetSymbolAddress) with
   the device current; make that first call before any stream capture.  The
   address is cached per CUDA context, so after a cudaDeviceReset the next
   call looks it up again (and that call, too, belongs outside a capture).
   All calls share the one array: calls whose work overlaps on the GPU (two
   streams, or two host threads) race and must not be issued.
   Sizes beyond the limits return RT_EINVAL with a message:
   1 <= N <= RT_ARNOLDI_STATIC_MAX_N, 0 <= j < RT_ARNOLDI_STATIC_MAX_J. */
#define RT_ARNOLDI_STATIC_MAX_N ((int64_t)1 << 40)
#define RT_ARNOLDI_STATIC_MAX_J 64
rt_status rt_arnoldi_mgs_static(double* V_dev, int64_t N, int32_t j, double* w_dev, double* h_dev, void* stream);

/* ---------------------------------------------------------------- solvers */
/* preconditioners.  NONE, JACOBI and LOCAL_LAMBDA are applied from the
   right (A M^-1 y = b, x = M^-1 y), so the stopping test is on the
   unpreconditioned residual.  JACOBI_LEFT (GMRES, FP64 only) solves
   D^-1 A x = D^-1 b and stops on the preconditioned residual, as the
   paper's experiments do (Sect. 4.2, Table 3).  For the sigma-form, JACOBI
   uses the diagonal of A (Eq. 18) and LOCAL_LAMBDA the inverse 2x2 blocks
   M_k = Id - J_k Lambda*_k T_k per height.

   SOR and SSOR (sigma-form only, FP64, 2*Ns <= 8192; Sect. 2.3): with
   A = D + L + U the assembled sigma-form matrix (unknowns interleaved per
   height, heights from the top), the upper SOR variant P = D/omega + U the
   paper's experiments use (Sect. 4.2), and the SSOR preconditioner
   P = omega/(2-omega) (D/omega + U) D^-1 (D/omega + L), whose inverse is a
   backward relaxation sweep followed by a forward one.  These readings
   reproduce Tables 4 and 5.  The first solve with a given (kind, omega)
   assembles A (2*Ns operator applies) and forms P^-1 densely on the device;
   each application is then one matrix-vector product, as the paper
   precomputes the action of P^-1.  SOR and SSOR are applied from the right
   (GMRES, BiCGSTAB, CGS) or as x <- x + P^-1 r (Richardson); SOR_LEFT and
   SSOR_LEFT precondition GMRES from the left, like JACOBI_LEFT. */
enum {
  RT_PREC_NONE = 0,
  RT_PREC_JACOBI = 1,
  RT_PREC_LOCAL_LAMBDA = 2,
  RT_PREC_JACOBI_LEFT = 3,
  RT_PREC_SOR = 4,
  RT_PREC_SSOR = 5,
  RT_PREC_SOR_LEFT = 6,
  RT_PREC_SSOR_LEFT = 7
};
/* Initial guess: zero, the caller's x_dev, or the paper's (Sect. 4.2: sigma
   = [1, 0, 1, 0, ...], i.e. sigma^0_0 = 1 and sigma^2_0 = 0 at every
   height).  For RT_FORM_SIGMA RT_X0_PAPER is that vector; for the I-form it
   is the radiation field that sigma produces, Lambda(T sigma) + t (Eq. 19):
   one formal solve with S_I = 1, S_Q = 0 and the boundary radiation.  The
   batch server always starts from zero. */
enum { RT_X0_ZERO = 0, RT_X0_USER = 1, RT_X0_PAPER = 2 };
enum { RT_ORTHO_MGS = 0, RT_ORTHO_CGS2 = 1 };
enum { RT_PRECISION_FP64 = 0, RT_PRECISION_FP32_REFINE = 1 };

typedef struct {
  int32_t restart;       /* GMRES restart length m, 1..160 (Sect. 2.1) */
  int32_t maxit;         /* cap on iterations (Arnoldi steps / BiCGSTAB-CGS iterations) */
  int32_t precond;       /* RT_PREC_*, applied from the right */
  int32_t x0_kind;       /* RT_X0_ZERO, RT_X0_USER (x_dev holds the initial guess) or RT_X0_PAPER */
  int32_t ortho;         /* GMRES Arnoldi: RT_ORTHO_MGS (default) or RT_ORTHO_CGS2 */
  int32_t precision;     /* RT_PRECISION_FP64, or FP32 operator inside FP64 iterative refinement */
  double rtol;           /* stop when ||b - A x||_2 / ||b||_2 < rtol (Sect. 4.2) */
  double inner_rtol;     /* FP32_REFINE: relative tolerance of each inner solve; <= 0: GMRES takes
                            rtol (each restart of its inner solve starts from the FP64 residual, so
                            one inner solve refines at every restart), BiCGSTAB/CGS 1e-4.  A step's
                            tolerance is at least rtol * ||b|| / ||r|| (no step over-solves) */
  int32_t max_refine;    /* FP32_REFINE: cap on refinement steps */
  double* resid_hist;    /* optional host array: relative residual estimate per iteration */
  int32_t hist_cap;      /* its capacity */
  double omega;          /* SOR / SSOR relaxation parameter, 0 < omega < 2 (Sect. 2.3) */
  double deadline_ms;    /* batch server only: a request not finished this long after its submission
                            ends with RT_ECANCELED (checked between restart cycles); 0: none */
} rt_solver_opts;

typedef struct {
  rt_status status;
  int32_t iters;         /* Arnoldi steps (GMRES) or full iterations (BiCGSTAB, CGS), all cycles */
  int32_t restarts;      /* GMRES cycles */
  int32_t applies;       /* products with A (FP64 and FP32) */
  int32_t refine_steps;  /* FP32_REFINE outer steps */
  int32_t hist_len;      /* entries written to resid_hist */
  double rel_resid;      /* final ||b - A x|| / ||b||, FP64 operator */
  double err_est;        /* the solver's own estimate of the same quantity when it stopped, without an
                            extra product: GMRES |g_{j+1}| / ||b|| of the last Arnoldi step (Givens
                            rotations, Sect. 2.1), BiCGSTAB / CGS the recursively updated residual,
                            Richardson the residual it formed; FP32_REFINE the last inner solve's
                            estimate times the outer relative residual it started from (what the FP64
                            residual would be with an exact FP32 operator); rel_resid when no step ran */
  double t_total_ms;     /* wall time of the call */
} rt_solve_info;

/* Fill opts with defaults: restart 30, maxit 10000, Jacobi, x0 = 0, MGS,
   FP64, rtol 1e-8, inner_rtol 0 (per solver, above), max_refine 20, no
   history, omega 1. */
void rt_solver_opts_default(rt_solver_opts* opts);

/* Right-preconditioned restarted GMRES(m) (Sect. 2.1; Saad & Schultz 1986),
   left-preconditioned with RT_PREC_JACOBI_LEFT, RT_PREC_SOR_LEFT or
   RT_PREC_SSOR_LEFT (then FP64 only; rel_resid is the preconditioned
   residual).  A cycle with m >= the steps needed is the
   paper's unrestarted GMRES.  With RT_PRECISION_FP32_REFINE the Arnoldi
   steps apply the FP32 operator and every restart cycle starts from the FP64
   residual b - A x; outer refinement steps (x += d, d from an inner solve to
   inner_rtol) wrap that.  b_dev, x_dev: N doubles.  Returns RT_OK when
   converged, RT_ENOTCONV at maxit, RT_EBREAKDOWN, RT_ENUMERIC; in each case
   x_dev holds the iterate. */
rt_status rt_solve_gmres(rt_problem* prob, const rt_solver_opts* opts, const double* b_dev,
                         double* x_dev, rt_solve_info* info, void* stream);
/* Right-preconditioned BiCGSTAB (Sect. 2.2; van der Vorst 1992); not with
   the left preconditioners.  With RT_PRECISION_FP32_REFINE the FP32 operator
   runs inside FP64 iterative refinement, as for GMRES: every outer step
   forms the FP64 residual, solves with the FP32 operator to inner_rtol and
   corrects x; iters counts the inner iterations of all steps. */
rt_status rt_solve_bicgstab(rt_problem* prob, const rt_solver_opts* opts, const double* b_dev,
                            double* x_dev, rt_solve_info* info, void* stream);
/* Right-preconditioned CGS (Sect. 2.2; Sonneveld 1989); not with the left
   preconditioners; RT_PRECISION_FP32_REFINE as for BiCGSTAB. */
rt_status rt_solve_cgs(rt_problem* prob, const rt_solver_opts* opts, const double* b_dev,
                       double* x_dev, rt_solve_info* info, void* stream);

/* Preconditioned Richardson iteration x <- x + M^-1 (b - A x) (Eq. 20); with
   the Jacobi preconditioner this is the Jacobi-Richardson (ALI) iteration the
   paper compares the Krylov solvers with (Sect. 2.3, Table 3).  Stops when
   ||b - A x|| / ||b|| < rtol (the unpreconditioned residual, computed every
   iteration) or after maxit updates; iters counts the updates.  FP64;
   preconditioners NONE, JACOBI, LOCAL_LAMBDA (either form), SOR and SSOR
   (sigma-form; the paper's SOR- and SSOR-Richardson rows of Tables 4-5). */
rt_status rt_solve_richardson(rt_problem* prob, const rt_solver_opts* opts, const double* b_dev,
                              double* x_dev, rt_solve_info* info, void* stream);

/* ----------------------------------------------------- batching and serving
   A server keeps many atmospheres resident on the device and solves them
   together by restarted GMRES(m) in lock-step: every phase of an Arnoldi step
   is one launch over all resident instances (the instances need not have the
   same sizes), and the whole restart cycle is one CUDA graph.  A worker
   thread admits submitted requests while a slot is free and the memory
   budget can hold the instance (tables, Krylov basis and work vectors in one
   device arena allocated at creation), runs cycles, and retires finished
   instances -- copying x to host memory and returning their memory -- before
   the next cycle, so requests that arrive while others are on the device join
   at the next cycle boundary (continuous batching).  Each instance's
   arithmetic depends only on its own data (deterministic reductions), so a
   result is the same whatever else is in the batch.  The problem is the one
   of rt_problem_create; the right-hand side is b = Lambda T c + t (rt_rhs)
   and the initial guess 0; the stopping rule is ||b - A x|| / ||b|| < rtol
   with the FP64 operator. */
typedef struct {
  int64_t mem_budget_bytes;  /* device arena for resident instances, allocated at creation */
  int32_t max_slots;         /* instances resident at once, 1..4096 */
  int32_t restart;           /* GMRES restart length for all instances, 1..160 (default 30; with the FP32
                                operator and the local-Lambda preconditioner 6..12 gave the most solves/s
                                on a batch of 512 uneven atmospheres) */
  int32_t precond;           /* RT_PREC_* for all instances */
  int32_t precision;         /* RT_PRECISION_FP64, or RT_PRECISION_FP32_REFINE: FP32 operator in the
                                Arnoldi steps, FP64 true residual at every restart (each restart is
                                an iterative-refinement step) */
  int32_t autotune;          /* 1: before the first cycle, time candidate grids of the persistent
                                kernels (quadrature, formal solver, vector passes) on the resident
                                instances and keep the fastest; 0: fixed grids.  Results do not
                                depend on the grids. */
  int32_t graphs;            /* 1: each restart cycle is one launch of a captured CUDA graph; 0: the
                                cycle's kernels are launched one by one on the server's stream (for
                                debugging and for tools that do not follow graphs).  Results are
                                the same either way. */
} rt_server_opts;

typedef struct rt_server rt_server;

/* defaults: 8 GiB budget, 64 slots, restart 30, local-Lambda, FP64, autotune on, graphs on */
void rt_server_opts_default(rt_server_opts* opts);
/* Create a server on the current device (the device stays the worker's). */
rt_status rt_server_create(const rt_server_opts* opts, rt_server** out);
/* rt_server_create with the server's device memory -- the arena of
   mem_budget_bytes that holds the resident instances, and the server's work
   lists and per-slot state -- requested from `allocator` (see rt_allocator).
   The functions and ctx must stay valid until rt_server_destroy has
   returned, which synchronises the device before the releases.  allocator
   NULL behaves as rt_server_create. */
rt_status rt_server_create_with_allocator(const rt_server_opts* opts, const rt_allocator* allocator,
                                          rt_server** out);
/* Queue one solve.  desc as for rt_problem_create (arrays copied; Ns <= 4096);
   opts may be NULL (rtol 1e-8, maxit 10000, no deadline) -- only rtol, maxit
   and deadline_ms are read.  *ticket identifies the request for rt_poll. */
rt_status rt_batch_submit(rt_server* srv, const rt_problem_desc* desc, const rt_solver_opts* opts,
                          uint64_t* ticket);
/* RT_EPENDING while the request is queued or resident; afterwards its final
   status (RT_OK, RT_ENOTCONV, RT_EBREAKDOWN, RT_ENUMERIC, RT_ENOMEM when the
   instance cannot fit the budget even alone, RT_ECANCELED), with info filled
   (t_total_ms: submission to completion) and, when x_host is not NULL, the
   N-vector solution copied there (the iterate reached, for a request ended
   by RT_ENOTCONV or RT_ECANCELED while resident; zeros for one that was
   never admitted).  A finished request is released by the poll that reports
   it. */
rt_status rt_poll(rt_server* srv, uint64_t ticket, rt_solve_info* info, double* x_host);

/* Cancel a request (no counterpart in the paper; a serving control).  A
   queued request ends at once; a resident one at the end of the restart
   cycle in progress, keeping the iterate it reached; either way rt_poll then
   reports RT_ECANCELED.  A request that already finished is left as it is.
   RT_OK, or RT_EINVAL for NULL or an unknown ticket (never issued, or
   already released by rt_poll).  Host only; thread-safe. */
rt_status rt_batch_cancel(rt_server* srv, uint64_t ticket);
typedef struct {
  int32_t resident;          /* instances on the device now */
  int32_t queued;            /* submitted, not yet admitted */
  int64_t arena_in_use;      /* bytes of the budget held by resident instances */
  int64_t arena_largest_free;/* largest contiguous free block of the budget */
  int64_t cycles;            /* restart cycles run so far */
  int64_t completed;         /* requests finished so far */
  int32_t grid_quad;         /* CTAs of the persistent quadrature kernel */
  int32_t grid_formal;       /* CTAs of the persistent formal-solver kernel */
  int32_t grid_vec;          /* CTAs of the persistent vector kernels */
  int32_t tuned;             /* 1 once the grids were autotuned */
} rt_server_stats;

/* Snapshot of the server's state (for monitoring). */
rt_status rt_server_stats_get(rt_server* srv, rt_server_stats* out);

/* Stop the worker (queued requests are dropped) and free everything. */
rt_status rt_server_destroy(rt_server* srv);

/* Thread-local message describing the last error returned on this thread. */
const char* rt_last_error(void);

/* Instrumentation (the paper has no counterpart; it counts this library's
   work): number of kernels this library has launched in the process so far.
   A kernel node of a captured CUDA graph counts once per graph launch. */
int64_t rt_launch_count(void);

/* Measurement aid (the paper has no counterpart): enqueues on `stream` one
   kernel that performs nothing but FP64 fused multiply-adds -- `iters`
   iterations of 8 independent chains per thread, 4 CTAs of 256 threads per
   SM -- and returns the number of FP64 floating-point operations it does
   (2 per fused multiply-add), or -1 (see rt_last_error) for iters < 1, a NULL
   sink_dev or a failed launch.  The caller times the launch with CUDA events
   on `stream`; FLOP / time is the FP64 rate that bounds the FP64 kernels of
   this library.  sink_dev: one caller-owned device double, overwritten (it
   keeps the chains from being optimised away). */
int64_t rt_probe_fp64_fma(int32_t iters, double* sink_dev, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* RT_KRYLOV_H */

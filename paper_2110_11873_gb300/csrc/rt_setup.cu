// Problem setup: discrete grids of Sect. 3.2 / 4.1 on the host, coefficient
// tables on the device, and the rt_problem_* entry points.
//
// Grids computed here (host, O(Nmu + Nnu) work):
//   * Gauss-Legendre nodes and weights by Newton's iteration on the Legendre
//     recurrence (full range on [-1,1], or per hemisphere on [0,1]);
//   * the Voigt function H(a,x) = Re w(x + i a) from Dawson's integral F(x)
//     (Rybicki's exponentially convergent sum) and the Taylor series of the
//     Faddeeva function w about the real axis:
//         w(x) = e^{-x^2} + (2i/sqrt(pi)) F(x),  w' = -2 z w + 2i/sqrt(pi),
//         w^{(n+1)} = -2 x w^{(n)} - 2 n w^{(n-1)},
//         H(a,x) = Re sum_n (i a)^n w^{(n)}(x) / n!;
//   * spectral weights: trapezoid x phi, optionally divided by their sum.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include <atomic>
#include <complex>
#include <mutex>
#include <unordered_map>

#include "rt_common.cuh"

namespace rt {

static thread_local std::string g_err;
thread_local int g_capturing = 0;
static std::atomic<long long> g_launch_count{0};
void count_launches(long long n) { g_launch_count.fetch_add(n, std::memory_order_relaxed); }

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
}
void clear_error() { g_err.clear(); }

// ------------------------------------------------------------ Gauss-Legendre
static void gauss_legendre(int n, std::vector<double>& t, std::vector<double>& w) {
  t.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = cos(M_PI * (i + 0.75) / (n + 0.5));  // near the (i+1)-th largest root
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-17) break;
    }
    {  // derivative at the converged root
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = (n == 1) ? 1.0 : n * (z * p1 - p0) / (z * z - 1.0);
    }
    double wt = 2.0 / ((1.0 - z * z) * dp * dp);
    t[i] = -z;
    t[n - 1 - i] = z;
    w[i] = wt;
    w[n - 1 - i] = wt;
  }
  if (n % 2 == 1) t[n / 2] = 0.0;
}

// ------------------------------------------------------------------- Voigt
// Dawson's integral F(x) = e^{-x^2} int_0^x e^{t^2} dt.
static double dawson(double x) {
  const double ax = fabs(x);
  if (ax < 0.2) {  // Maclaurin series: sum (-1)^n 2^n x^{2n+1} / (2n+1)!!
    double term = x, sum = x, x2 = x * x;
    for (int n = 1; n < 30; ++n) {
      term *= -2.0 * x2 / (2.0 * n + 1.0);
      sum += term;
      if (fabs(term) < 1e-18 * fabs(sum)) break;
    }
    return sum;
  }
  // Rybicki: F(x) = lim_{h->0} pi^{-1/2} sum_{n odd} e^{-(x - n h)^2} / n; the
  // error of step h decays like exp(-(pi/(2h))^2), ~1e-27 at h = 0.2.  The sum
  // is centred on the even index n0 nearest x/h.
  const double h = 0.2;
  const int n0 = 2 * (int)lround(ax / (2.0 * h));
  const double xp = ax - n0 * h;
  double s = 0.0;
  for (int j = -24; j < 24; ++j) {
    const int n = 2 * j + 1;
    const double d = xp - n * h;
    s += exp(-d * d) / (double)(n + n0);
  }
  s /= sqrt(M_PI);
  return x < 0 ? -s : s;
}

static double voigt_H(double a, double x) {
  typedef std::complex<double> C;
  const double rsp = 1.0 / sqrt(M_PI);
  C w0(exp(-x * x), 2.0 * rsp * dawson(x));
  C w1 = -2.0 * x * w0 + C(0.0, 2.0 * rsp);
  C ia(0.0, a), pw(1.0, 0.0);
  double sum = w0.real();
  C wn = w1, wprev = w0;
  double fact = 1.0;
  for (int n = 1; n < 80; ++n) {
    fact *= n;
    pw *= ia;
    C term = pw * wn / fact;
    sum += term.real();
    if (n > 3 && std::abs(term) < 1e-19 * fabs(sum)) break;
    C wnext = -2.0 * x * wn - 2.0 * n * wprev;
    wprev = wn;
    wn = wnext;
  }
  return sum;
}

// ------------------------------------------------------------ validation
rt_status validate_desc(const rt_problem_desc* d) {
  if (!d) { set_error("desc is NULL"); return RT_EINVAL; }
  if (d->Ns < 2) { set_error("Ns must be >= 2 (got %d)", d->Ns); return RT_EINVAL; }
  if (d->Nmu < 2 || d->Nmu % 2 || d->Nmu > 256) {
    set_error("Nmu must be even and in [2,256] (got %d)", d->Nmu);
    return RT_EINVAL;
  }
  if (d->Nnu < 2) { set_error("Nnu must be >= 2 (got %d)", d->Nnu); return RT_EINVAL; }
  if (!d->tau) { set_error("tau is required"); return RT_EINVAL; }
  for (int k = 0; k + 1 < d->Ns; ++k)
    if (!(d->tau[k + 1] > d->tau[k])) { set_error("tau must be strictly increasing (k=%d)", k); return RT_EINVAL; }
  if (!(d->eps > 0.0 && d->eps <= 1.0)) { set_error("eps must lie in (0,1]"); return RT_EINVAL; }
  if (!(d->a > 0.0)) { set_error("a must be > 0"); return RT_EINVAL; }
  if (!(d->x_max > d->x_min)) { set_error("x_min must be < x_max"); return RT_EINVAL; }
  if (!d->phi) {
    if (d->a > 0.1) { set_error("internal Voigt profile needs a <= 0.1; pass phi"); return RT_EINVAL; }
    if (fabs(d->x_min) > 12.0 || fabs(d->x_max) > 12.0) {
      set_error("internal Voigt profile needs |x| <= 12; pass phi");
      return RT_EINVAL;
    }
  } else if (d->tau_kind == RT_TAU_LINE_CENTER && !(d->phi_center > 0.0)) {
    set_error("phi_center must be > 0 when phi is given with line-centre tau");
    return RT_EINVAL;
  }
  if (d->tau_kind != RT_TAU_LINE_CENTER && d->tau_kind != RT_TAU_FREQ_INTEGRATED) { set_error("bad tau_kind"); return RT_EINVAL; }
  if (d->mu_quad != RT_MU_GL_HALF && d->mu_quad != RT_MU_GL_FULL) { set_error("bad mu_quad"); return RT_EINVAL; }
  if (d->formal_solver < RT_FS_DELO_LINEAR || d->formal_solver > RT_FS_DELO_PARABOLIC) { set_error("bad formal_solver"); return RT_EINVAL; }
  if (d->form != RT_FORM_I && d->form != RT_FORM_SIGMA) { set_error("bad form"); return RT_EINVAL; }
  const int64_t N = 2LL * d->Ns * d->Nmu * d->Nnu;
  if (N > (int64_t)1 << 34) { set_error("problem too large (N=%lld)", (long long)N); return RT_EINVAL; }
  return RT_OK;
}

void host_grids(const rt_problem_desc* d, Problem& P) {
  P.Ns = d->Ns; P.Nmu = d->Nmu; P.Nnu = d->Nnu; P.Nh = d->Nmu / 2;
  P.nray = (int64_t)d->Nmu * d->Nnu;
  P.N = 2 * (int64_t)d->Ns * P.nray;
  P.form = d->form;
  P.Nop = d->form == RT_FORM_SIGMA ? 2 * (int64_t)d->Ns : P.N;
  P.eps = d->eps; P.xi = 1.0 - d->eps; P.W2 = d->W2; P.a = d->a;
  P.tau_kind = d->tau_kind; P.mu_quad = d->mu_quad; P.fs = d->formal_solver;
  P.freq_norm = d->freq_norm;
  P.tau.assign(d->tau, d->tau + d->Ns);
  if (d->B) P.B.assign(d->B, d->B + d->Ns); else P.B.assign(d->Ns, 1.0);
  // directions, ascending
  const int Nh = P.Nh;
  P.mu.assign(P.Nmu, 0.0);
  P.w_mu.assign(P.Nmu, 0.0);
  std::vector<double> t, w;
  if (d->mu_quad == RT_MU_GL_FULL) {
    gauss_legendre(P.Nmu, t, w);
    P.mu = t;
    P.w_mu = w;
  } else {
    gauss_legendre(Nh, t, w);  // ascending on [-1,1]
    for (int i = 0; i < Nh; ++i) {
      const double mp = 0.5 * (t[i] + 1.0), wp = 0.5 * w[i];
      P.mu[Nh + i] = mp;
      P.w_mu[Nh + i] = wp;
      P.mu[Nh - 1 - i] = -mp;
      P.w_mu[Nh - 1 - i] = wp;
    }
  }
  const double s2 = sqrt(2.0);
  P.t201.resize(P.Nmu);
  P.t202.resize(P.Nmu);
  for (int m = 0; m < P.Nmu; ++m) {
    const double m2 = P.mu[m] * P.mu[m];
    P.t201[m] = s2 * (3.0 * m2 - 1.0) / 4.0;
    P.t202[m] = s2 * (3.0 * m2 - 3.0) / 4.0;
  }
  // frequencies, profile, weights
  const int Nnu = P.Nnu;
  const double h = (d->x_max - d->x_min) / (Nnu - 1);
  P.x.resize(Nnu);
  P.phi.resize(Nnu);
  P.w_nu.resize(Nnu);
  P.phi_hat.resize(Nnu);
  for (int p = 0; p < Nnu; ++p) P.x[p] = (p == Nnu - 1) ? d->x_max : d->x_min + p * h;
  double phi_c;
  if (d->phi) {
    for (int p = 0; p < Nnu; ++p) P.phi[p] = d->phi[p];
    phi_c = d->phi_center;
  } else {
    const double rsp = 1.0 / sqrt(M_PI);
    for (int p = 0; p < Nnu; ++p) P.phi[p] = voigt_H(d->a, P.x[p]) * rsp;
    phi_c = voigt_H(d->a, 0.0) * rsp;
  }
  double wsum = 0.0;
  for (int p = 0; p < Nnu; ++p) {
    const double c = (p == 0 || p == Nnu - 1) ? 0.5 * h : h;
    P.w_nu[p] = c * P.phi[p];
    wsum += P.w_nu[p];
  }
  if (d->freq_norm)
    for (int p = 0; p < Nnu; ++p) P.w_nu[p] /= wsum;
  for (int p = 0; p < Nnu; ++p)
    P.phi_hat[p] = (d->tau_kind == RT_TAU_LINE_CENTER) ? P.phi[p] / phi_c : P.phi[p];
}


namespace {
class HookAlloc : public DevAllocator {
 public:
  HookAlloc(const rt_allocator& h, cudaStream_t st) : h_(h), st_(st) {}
  cudaError_t alloc(void** p, size_t bytes) override {
    *p = nullptr;
    if (bytes == 0) bytes = 256;
    void* q = h_.alloc(h_.ctx, bytes, reinterpret_cast<void*>(st_));
    if (!q) return cudaErrorMemoryAllocation;
    if (reinterpret_cast<uintptr_t>(q) & 255) {   // the kernels assume 256-byte aligned blocks
      h_.release(h_.ctx, q, bytes, reinterpret_cast<void*>(st_));
      return cudaErrorMemoryAllocation;
    }
    {
      std::lock_guard<std::mutex> lk(mu_);
      sizes_[q] = bytes;
    }
    *p = q;
    return cudaSuccess;
  }
  void release(void* p) override {
    if (!p) return;
    size_t bytes = 0;
    {
      std::lock_guard<std::mutex> lk(mu_);
      auto it = sizes_.find(p);
      if (it == sizes_.end()) return;
      bytes = it->second;
      sizes_.erase(it);
    }
    h_.release(h_.ctx, p, bytes, reinterpret_cast<void*>(st_));
  }

 private:
  rt_allocator h_;
  cudaStream_t st_;
  std::mutex mu_;
  std::unordered_map<void*, size_t> sizes_;
};
}  // namespace

DevAllocator* make_hook_allocator(const rt_allocator* hook, cudaStream_t st) {
  if (!hook || !hook->alloc || !hook->release) return nullptr;
  return new (std::nothrow) HookAlloc(*hook, st);
}

}  // namespace rt

using namespace rt;

static rt_status create_problem(const rt_problem_desc* desc, const rt_allocator* hook, void* stream,
                                rt_problem** out) {
  RT_NVTX("rt_problem_create");
  clear_error();
  if (!out) { set_error("out is NULL"); return RT_EINVAL; }
  *out = nullptr;
  RT_TRY(validate_desc(desc));
  if (hook && (!hook->alloc || !hook->release)) {
    set_error("the allocator needs both alloc and release");
    return RT_EINVAL;
  }
  rt_problem* pr = new (std::nothrow) rt_problem();
  if (!pr) { set_error("host allocation failed"); return RT_ENOMEM; }
  Problem& P = pr->P;
  if (hook) {
    P.own_alloc = make_hook_allocator(hook, as_stream(stream));
    if (!P.own_alloc) {
      delete pr;
      set_error("host allocation failed");
      return RT_ENOMEM;
    }
    P.alloc = P.own_alloc;
  }
  host_grids(desc, P);
  cudaError_t e = cudaGetDevice(&P.device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&P.num_sms, cudaDevAttrMultiProcessorCount, P.device);
  if (e != cudaSuccess) {
    set_error("no CUDA device: %s", cudaGetErrorString(e));
    delete P.own_alloc;
    delete pr;
    return RT_ECUDA;
  }
  rt_status s = setup_device_tables(&P, as_stream(stream));
  if (s != RT_OK) {
    if (P.own_alloc) cudaDeviceSynchronize();
    free_device(&P);
    delete P.own_alloc;
    delete pr;
    return s;
  }
  *out = pr;
  return RT_OK;
}

extern "C" {

const char* rt_last_error(void) { return rt::g_err.c_str(); }

int64_t rt_launch_count(void) { return (int64_t)rt::g_launch_count.load(std::memory_order_relaxed); }

rt_status rt_problem_create(const rt_problem_desc* desc, void* stream, rt_problem** out) {
  return create_problem(desc, nullptr, stream, out);
}

rt_status rt_problem_create_with_allocator(const rt_problem_desc* desc, const rt_allocator* allocator, void* stream,
                                           rt_problem** out) {
  return create_problem(desc, allocator, stream, out);
}

rt_status rt_problem_destroy(rt_problem* prob) {
  RT_NVTX("rt_problem_destroy");
  if (!prob) return RT_OK;
  release_graphs(&prob->P);
  // a caller's allocator may hand a released block to its next user at once:
  // nothing of this problem may still be running on the device
  if (prob->P.own_alloc) cudaDeviceSynchronize();
  free_device(&prob->P);
  delete prob->P.own_alloc;
  delete prob;
  return RT_OK;
}

int64_t rt_problem_size(const rt_problem* prob) { return prob ? prob->P.Nop : -1; }

rt_status rt_problem_check(rt_problem* prob, void* stream) {
  clear_error();
  if (!prob) { set_error("prob is NULL"); return RT_EINVAL; }
  return check_device_flag(&prob->P, as_stream(stream));
}

int rt_problem_formal_kernel(const rt_problem* prob) { return prob ? prob->P.staged : -1; }

rt_status rt_problem_inject_wait_timeout(rt_problem* prob, int32_t count) {
  clear_error();
  if (!prob || count < 0) {
    set_error("prob is NULL or count < 0");
    return RT_EINVAL;
  }
  prob->P.inject_wait_fail = count;
  return RT_OK;
}

rt_status rt_problem_grids(const rt_problem* prob, double* mu, double* w_mu, double* x,
                           double* phi, double* w_nu, double* phi_hat) {
  if (!prob) { set_error("prob is NULL"); return RT_EINVAL; }
  const Problem& P = prob->P;
  for (int m = 0; m < P.Nmu; ++m) {
    if (mu) mu[m] = P.mu[m];
    if (w_mu) w_mu[m] = P.w_mu[m];
  }
  for (int p = 0; p < P.Nnu; ++p) {
    if (x) x[p] = P.x[p];
    if (phi) phi[p] = P.phi[p];
    if (w_nu) w_nu[p] = P.w_nu[p];
    if (phi_hat) phi_hat[p] = P.phi_hat[p];
  }
  return RT_OK;
}

}  // extern "C"

// Host float64 construction of the CP Newton kernel: sinc-quadrature nodes
// (Appendix 3, Eq. sinc_Newt) and Galerkin cell integrals (Appendix 3,
// Eq. galten), plus the FFT twiddle tables.  The device part of
// make_newton_kernel (spectra) lives in spectra.cu.
#include <cmath>
#include <cstring>
#include <mutex>

#include "cpc_internal.h"

namespace cpc {

namespace {
thread_local std::string g_last_error;
const double kPi = 3.14159265358979323846;
}  // namespace

int fail(int status, const std::string& msg) {
  g_last_error = msg;
  return status;
}
int cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return CPC_ERR_CUDA;
}
void clear_error() { g_last_error.clear(); }
const char* last_error() { return g_last_error.c_str(); }

// ---- sinc rule -------------------------------------------------------------
// 1/r = (2/sqrt(pi)) int_R exp(-e^{2u} r^2) e^u du, trapezoid in u with 2M+1
// nodes u0 + k hs.  Three error estimates (natural logs) are balanced:
//   discretisation   ld  = ln(2 sqrt2) - pi^2/(2 hs)
//   far truncation   llo = ln((2/sqrt(pi)) hs r_max) + u0 - M hs - hs - ln(1 - e^{-hs})
//   near truncation  lhi = ln(2 pi hs/(1 - e^{-2hs}) / cell) - 2(u0 + M hs + hs),
// where cell is the Galerkin entry of the cell(s) touching the origin:
// 2 kappa h^2 for the centred convolution grid, 8 kappa h^2 for the master
// grid (origin on a corner shared by 8 cells of kappa h^2, each getting 1/8
// of a narrow Gaussian), kappa = int_{[0,1]^3} |x|^-1 dx.
static void rule_logs(int M, double hs, double u0, double h, double r_max, bool master,
                      double* llo, double* lhi, double* ld) {
  const double kappa = 3.0 * std::log((1.0 + std::sqrt(3.0)) / std::sqrt(2.0)) - kPi / 4.0;
  const double cell = (master ? 8.0 : 2.0) * kappa * h * h;
  *llo = std::log(2.0 / std::sqrt(kPi) * hs * r_max) + (u0 - M * hs) - hs -
         std::log(-std::expm1(-hs));
  *lhi = std::log(2.0 * kPi * hs / -std::expm1(-2.0 * hs) / cell) - 2.0 * (u0 + M * hs + hs);
  *ld = std::log(2.0 * std::sqrt(2.0)) - kPi * kPi / (2.0 * hs);
}

static double shift_for_step(int M, double hs, double h, double r_max, bool master) {
  double lo = -200.0, hi = 200.0;
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi), a, c, d;
    rule_logs(M, hs, mid, h, r_max, master, &a, &c, &d);
    if (a > c) hi = mid; else lo = mid;
  }
  return 0.5 * (lo + hi);
}

void sinc_rule(int M, double h, double r_max, bool master, double* hs_out, double* u0_out) {
  double lo = 0.02, hi = 3.0;
  for (int it = 0; it < 200; ++it) {
    double hs = 0.5 * (lo + hi);
    double u0 = shift_for_step(M, hs, h, r_max, master);
    double a, c, d;
    rule_logs(M, hs, u0, h, r_max, master, &a, &c, &d);
    if (d > a) hi = hs; else lo = hs;
  }
  *hs_out = 0.5 * (lo + hi);
  *u0_out = shift_for_step(M, *hs_out, h, r_max, master);
}

// ---- cell integrals ----------------------------------------------------------
// int_{x0}^{x1} exp(-t^2 x^2) dx.  Narrow cells relative to the Gaussian
// (t (x1-x0) < 1/16) use 16-point Gauss-Legendre (nodes by Newton iteration
// on P_16); otherwise erf/erfc differences on the positive side, erfc when
// the cell starts beyond t x = 1/2 (no cancellation near erf -> 1).
namespace {
struct GaussLegendre16 {
  double x[16], w[16];
  // P_16 and P_15 at z by the three-term recurrence
  static void legendre(double z, double* pm, double* pm1) {
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= 16; ++k) {
      const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    *pm = p1;
    *pm1 = p0;
  }
  GaussLegendre16() {
    const int m = 16;
    for (int i = 0; i < m; ++i) {
      double z = std::cos(kPi * (i + 0.75) / (m + 0.5));
      for (int it = 0; it < 50; ++it) {
        double pm, pm1;
        legendre(z, &pm, &pm1);
        const double dp = m * (z * pm - pm1) / (z * z - 1.0);
        const double dz = pm / dp;
        z -= dz;
        if (std::fabs(dz) <= 1e-16 * std::fabs(z)) break;
      }
      double pm, pm1;
      legendre(z, &pm, &pm1);
      const double dp = m * (z * pm - pm1) / (z * z - 1.0);
      x[i] = z;
      w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
  }
};
const GaussLegendre16& gl16() {
  static GaussLegendre16 g;
  return g;
}
}  // namespace

double gauss_cell_integral(double t, double x0, double x1) {
  const double width = x1 - x0;
  if (t * width < 0.0625) {
    const GaussLegendre16& g = gl16();
    const double mid = 0.5 * (x0 + x1), half = 0.5 * width;
    double s = 0.0;
    for (int i = 0; i < 16; ++i) {
      const double y = t * (mid + half * g.x[i]);
      s += g.w[i] * std::exp(-y * y);
    }
    return half * s;
  }
  const double scale = std::sqrt(kPi) / (2.0 * t);
  double lo = x0, hi = x1;
  if (hi <= 0.0) { lo = -x1; hi = -x0; }
  if (lo * t >= 0.5) return scale * (std::erfc(t * lo) - std::erfc(t * hi));
  return scale * (std::erf(t * hi) - std::erf(t * lo));
}

// ---- twiddles ------------------------------------------------------------------
// cos/sin of 2 pi e / N: the angle is split into the nearest quarter turn
// m pi/2 (exact sign/swap) and a remainder |d| <= pi/4 formed from an exact
// integer numerator, so the only rounding is in cos(d), sin(d).
static void unit_root(long e, long N, double* c, double* s) {
  e %= N;
  if (e < 0) e += N;
  const long m = (4 * e + N / 2) / N;
  const double d = double(4 * e - m * N) / double(N) * (kPi / 2.0);
  const double cd = std::cos(d), sd = std::sin(d);
  switch (m & 3) {
    case 0: *c = cd; *s = sd; break;
    case 1: *c = -sd; *s = cd; break;
    case 2: *c = -cd; *s = -sd; break;
    default: *c = sd; *s = -cd; break;
  }
}

void build_twiddles(int n, std::vector<double>& tw_re, std::vector<double>& tw_im,
                    std::vector<double>& hw_re, std::vector<double>& hw_im) {
  tw_re.resize(n); tw_im.resize(n);
  for (int e = 0; e < n; ++e) {
    double c, s;
    unit_root(e, n, &c, &s);
    tw_re[e] = c; tw_im[e] = -s;   // exp(-2 pi i e/n)
  }
  hw_re.resize(n + 1); hw_im.resize(n + 1);
  for (int f = 0; f <= n; ++f) {
    double c, s;
    unit_root(f, 2L * n, &c, &s);
    hw_re[f] = c; hw_im[f] = -s;   // exp(-2 pi i f/(2n))
  }
}

}  // namespace cpc

using namespace cpc;

extern "C" {

const char* cpc_status_string(int status) {
  switch (status) {
    case CPC_OK: return "ok";
    case CPC_ERR_INVALID: return "invalid argument";
    case CPC_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case CPC_ERR_CUDA: return "CUDA runtime error";
    case CPC_ERR_DEVICE: return "device-side check failed";
    case CPC_ERR_UNSUPPORTED: return "unsupported size or precision";
    default: return "unknown status";
  }
}

const char* cpc_last_error(void) { return cpc::last_error(); }

static int validate_kernel_args(int n, double b, int M, int kind, const char* who) {
  if (!is_pow2(n) || n < 16 || n > 16384)
    return fail(CPC_ERR_UNSUPPORTED, std::string(who) + ": n must be a power of two in [16, 16384]");
  if (kind == CPC_KERNEL_CONV && n > 8192)
    return fail(CPC_ERR_UNSUPPORTED, std::string(who) + ": convolution kernels support n <= 8192");
  if (!(b > 0.0) || !std::isfinite(b)) return fail(CPC_ERR_INVALID, std::string(who) + ": b must be > 0");
  if (M < 1 || M > 64) return fail(CPC_ERR_INVALID, std::string(who) + ": M must be in [1, 64]");
  if (kind != CPC_KERNEL_CONV && kind != CPC_KERNEL_MASTER)
    return fail(CPC_ERR_INVALID, std::string(who) + ": unknown kind");
  return CPC_OK;
}

// nodes, weights and Galerkin vectors on the host (float64)
static void host_tables(cpc_kernel* P) {
  const bool master = (P->kind == CPC_KERNEL_MASTER);
  sinc_rule(P->M, P->h, 2.0 * std::sqrt(3.0) * P->b, master, &P->hs, &P->u0);
  P->t.resize(P->R_N);
  P->a.resize(P->R_N);
  for (int q = 0; q < P->R_N; ++q) {
    const int k = q - P->M;
    P->t[q] = std::exp(P->u0 + k * P->hs);
    P->a[q] = 2.0 / std::sqrt(kPi) * P->hs * P->t[q];
  }
  P->p.assign(size_t(P->R_N) * P->len, 0.0);
  const double h = P->h;
  const int n = P->n;
  for (int q = 0; q < P->R_N; ++q) {
    const double scale = std::cbrt(P->a[q]);
    double* row = &P->p[size_t(q) * P->len];
    if (!master) {
      for (int m = 0; m < n; ++m) row[m] = scale * gauss_cell_integral(P->t[q], (m - 0.5) * h, (m + 0.5) * h);
    } else {
      for (int j = -n; j < n; ++j) row[j + n] = scale * gauss_cell_integral(P->t[q], j * h, (j + 1.0) * h);
    }
  }
}

int make_newton_kernel_tables(int n, double b, int M, int kind, double* t, double* a, double* p,
                              double* hs, double* u0) {
  clear_error();
  int st = validate_kernel_args(n, b, M, kind, "make_newton_kernel_tables");
  if (st) return st;
  cpc_kernel K;
  K.n = n; K.b = b; K.h = 2.0 * b / n; K.M = M; K.R_N = 2 * M + 1; K.kind = kind;
  K.len = (kind == CPC_KERNEL_CONV) ? n : 2 * n;
  host_tables(&K);
  if (t) std::memcpy(t, K.t.data(), sizeof(double) * K.R_N);
  if (a) std::memcpy(a, K.a.data(), sizeof(double) * K.R_N);
  if (p) std::memcpy(p, K.p.data(), sizeof(double) * K.p.size());
  if (hs) *hs = K.hs;
  if (u0) *u0 = K.u0;
  return CPC_OK;
}

// the host path plan of a CONV kernel of make_newton_kernel(n, b, M), with no
// device work (make_newton_kernel_paths, make_newton_kernel_eh_plan)
static int host_plan(int n, double b, int M, int max_half_width32, int max_half_width64, int max_rank32,
                     int max_rank64, const char* who, cpc_kernel& K, TermPlan& tp) {
  int st = validate_kernel_args(n, b, M, CPC_KERNEL_CONV, who);
  if (st) return st;
  if (max_half_width32 < -1 || max_half_width32 > 32 || max_half_width64 < -1 || max_half_width64 > 32 ||
      max_rank32 < -1 || max_rank32 > 16 || max_rank64 < -1 || max_rank64 > 16)
    return fail(CPC_ERR_INVALID, std::string(who) + ": half-widths in [-1, 32], ranks in [-1, 16]");
  K.n = n; K.b = b; K.h = 2.0 * b / n; K.M = M; K.R_N = 2 * M + 1; K.kind = CPC_KERNEL_CONV;
  K.len = n;
  host_tables(&K);
  plan_term_paths(&K, max_half_width32, max_half_width64, max_rank32, max_rank64, tp);
  return CPC_OK;
}

int make_newton_kernel_eh_plan(int n, double b, int M, int max_half_width32, int max_half_width64, int max_rank32,
                               int max_rank64, int* plan) {
  clear_error();
  if (!plan) return fail(CPC_ERR_INVALID, "make_newton_kernel_eh_plan: plan is NULL");
  cpc_kernel K;
  TermPlan tp;
  int st = host_plan(n, b, M, max_half_width32, max_half_width64, max_rank32, max_rank64,
                     "make_newton_kernel_eh_plan", K, tp);
  if (st) return st;
  for (int cls = 0; cls < 2; ++cls) {
    plan[3 * cls] = tp.n_lag[cls];
    plan[3 * cls + 1] = tp.n_cov[cls];
    plan[3 * cls + 2] = tp.n_eh[cls];
  }
  return CPC_OK;
}

int make_newton_kernel_paths(int n, double b, int M, int max_half_width32, int max_half_width64, int max_rank32,
                             int max_rank64, int* half_width, int* rank, double* cheb) {
  clear_error();
  cpc_kernel K;
  TermPlan tp;
  int st = host_plan(n, b, M, max_half_width32, max_half_width64, max_rank32, max_rank64,
                     "make_newton_kernel_paths", K, tp);
  if (st) return st;
  for (int cls = 0; cls < 2; ++cls)
    for (int q = 0; q < K.R_N; ++q) {
      if (half_width) half_width[cls * K.R_N + q] = tp.terms[size_t(cls) * kTermRows * K.R_N + q];
      if (rank) rank[cls * K.R_N + q] = tp.terms[size_t(cls) * kTermRows * K.R_N + K.R_N + q];
    }
  if (cheb) std::memcpy(cheb, tp.cheb.data(), sizeof(double) * tp.cheb.size());
  return CPC_OK;
}

int make_newton_kernel(int n, double b, int M, int kind, void* stream, cpc_kernel** out) {
  clear_error();
  if (!out) return fail(CPC_ERR_INVALID, "make_newton_kernel: out is NULL");
  *out = nullptr;
  int st0 = validate_kernel_args(n, b, M, kind, "make_newton_kernel");
  if (st0) return st0;

  cpc_kernel* P = new cpc_kernel();
  P->n = n; P->b = b; P->h = 2.0 * b / n; P->M = M; P->R_N = 2 * M + 1; P->kind = kind;
  P->len = (kind == CPC_KERNEL_CONV) ? n : 2 * n;
  const bool master = (kind == CPC_KERNEL_MASTER);
  host_tables(P);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int st = CPC_OK;
  auto cleanup = [&]() { cpc_kernel_free(P); };
  cudaError_t e = cudaMalloc(&P->d_p, sizeof(double) * P->p.size());
  if (e == cudaSuccess) e = cudaMemcpyAsync(P->d_p, P->p.data(), sizeof(double) * P->p.size(), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) { st = cuda_fail(e, "make_newton_kernel: table upload"); cleanup(); return st; }
  if (master) {
    e = cudaMalloc(&P->d_lat, lattice_scratch_bytes(n));
    if (e != cudaSuccess) { st = cuda_fail(e, "make_newton_kernel: lattice scratch"); cleanup(); return st; }
  }
  if (!master) {
    std::vector<double> twr, twi, hwr, hwi;
    build_twiddles(n, twr, twi, hwr, hwi);
    std::vector<double2> tw64(n), hw64(n + 1);
    std::vector<float2> tw32(n), hw32(n + 1);
    for (int i = 0; i < n; ++i) { tw64[i] = make_double2(twr[i], twi[i]); tw32[i] = make_float2(float(twr[i]), float(twi[i])); }
    for (int i = 0; i <= n; ++i) { hw64[i] = make_double2(hwr[i], hwi[i]); hw32[i] = make_float2(float(hwr[i]), float(hwi[i])); }
    e = cudaMalloc(&P->d_tw64, sizeof(double2) * n);
    if (e == cudaSuccess) e = cudaMalloc(&P->d_tw32, sizeof(float2) * n);
    if (e == cudaSuccess) e = cudaMalloc(&P->d_hw64, sizeof(double2) * (n + 1));
    if (e == cudaSuccess) e = cudaMalloc(&P->d_hw32, sizeof(float2) * (n + 1));
    if (e == cudaSuccess) e = cudaMalloc(&P->d_phat64, sizeof(double) * size_t(P->R_N) * (n + 1));
    if (e == cudaSuccess) e = cudaMalloc(&P->d_phat32, sizeof(float) * size_t(P->R_N) * (n + 1));
    if (e == cudaSuccess) e = cudaMemcpyAsync(P->d_tw64, tw64.data(), sizeof(double2) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(P->d_tw32, tw32.data(), sizeof(float2) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(P->d_hw64, hw64.data(), sizeof(double2) * (n + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(P->d_hw32, hw32.data(), sizeof(float2) * (n + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMalloc(&P->d_twp64, sizeof(double2) * n);
    if (e == cudaSuccess) e = cudaMalloc(&P->d_twp32, sizeof(float2) * n);
    if (e == cudaSuccess) e = cudaMalloc(&P->d_twp32_lo, 4 * size_t(n));
    if (e == cudaSuccess) e = cudaMalloc(&P->d_hw32_lo, 4 * size_t(n + 1));
    if (e == cudaSuccess) e = cudaMalloc(&P->d_pp32, sizeof(float2) * size_t(P->R_N) * n);
    if (e == cudaSuccess) e = cudaMalloc(&P->d_opf32, sizeof(float4) * size_t(n));
    if (e != cudaSuccess) { st = cuda_fail(e, "make_newton_kernel: FFT tables"); cleanup(); return st; }
    st = build_pass_twiddles(P, s);
    if (st != CPC_OK) { cleanup(); return st; }
    st = compute_kernel_spectrum(P, s);
    if (st != CPC_OK) { cleanup(); return st; }
    st = build_kernel_pairs(P, s);
    if (st != CPC_OK) { cleanup(); return st; }
    e = cudaMalloc(&P->d_specw32, sizeof(float) * size_t(P->R_N) * 2 * (n + 1));
    if (e != cudaSuccess) { st = cuda_fail(e, "make_newton_kernel: spectral weights"); cleanup(); return st; }
    st = build_spectral_weights(P, P->d_specw32, s);
    if (st != CPC_OK) { cleanup(); return st; }
    st = build_term_tables(P, kDefaultBand32, kDefaultBand64, kDefaultRank, kDefaultRank, s);
    if (st != CPC_OK) { cleanup(); return st; }
    st = build_df_tables(P, s);
    if (st != CPC_OK) { cleanup(); return st; }
  }
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) { st = cuda_fail(e, "make_newton_kernel: synchronize"); cleanup(); return st; }
  *out = P;
  return CPC_OK;
}

int cpc_kernel_info(const cpc_kernel* P, int* n, double* b, int* M, int* R_N, int* kind,
                    double* hs, double* u0) {
  if (!P) return fail(CPC_ERR_INVALID, "cpc_kernel_info: NULL kernel");
  if (n) *n = P->n;
  if (b) *b = P->b;
  if (M) *M = P->M;
  if (R_N) *R_N = P->R_N;
  if (kind) *kind = P->kind;
  if (hs) *hs = P->hs;
  if (u0) *u0 = P->u0;
  return CPC_OK;
}

int cpc_kernel_tables(const cpc_kernel* P, double* t, double* a, double* p) {
  if (!P) return fail(CPC_ERR_INVALID, "cpc_kernel_tables: NULL kernel");
  if (t) std::memcpy(t, P->t.data(), sizeof(double) * P->R_N);
  if (a) std::memcpy(a, P->a.data(), sizeof(double) * P->R_N);
  if (p) std::memcpy(p, P->p.data(), sizeof(double) * P->p.size());
  return CPC_OK;
}

int cpc_kernel_set_conv_paths(cpc_kernel* P, int max_half_width32, int max_half_width64, int max_rank32,
                              int max_rank64, void* stream) {
  clear_error();
  if (!P) return fail(CPC_ERR_INVALID, "cpc_kernel_set_conv_paths: NULL kernel");
  if (P->kind != CPC_KERNEL_CONV) return fail(CPC_ERR_INVALID, "cpc_kernel_set_conv_paths: needs a CONV kernel");
  if (max_half_width32 < -1 || max_half_width32 > 32 || max_half_width64 < -1 || max_half_width64 > 32)
    return fail(CPC_ERR_INVALID, "cpc_kernel_set_conv_paths: half-widths must lie in [-1, 32]");
  if (max_rank32 < -1 || max_rank32 > 16 || max_rank64 < -1 || max_rank64 > 16)
    return fail(CPC_ERR_INVALID, "cpc_kernel_set_conv_paths: ranks must lie in [-1, 16]");
  return build_term_tables(P, max_half_width32, max_half_width64, max_rank32, max_rank64,
                           static_cast<cudaStream_t>(stream));
}

int cpc_kernel_conv_paths(const cpc_kernel* P, int precision, int* half_width, int* rank) {
  clear_error();
  if (!P) return fail(CPC_ERR_INVALID, "cpc_kernel_conv_paths: NULL kernel");
  if (!known_precision(precision)) return fail(CPC_ERR_UNSUPPORTED, "cpc_kernel_conv_paths: unknown precision form");
  const int cls = storage_precision(precision) == CPC_FP32 ? 0 : 1;
  const bool conv = P->kind == CPC_KERNEL_CONV;
  for (int q = 0; q < P->R_N; ++q) {
    if (half_width) half_width[q] = (conv && !P->band_h[cls].empty()) ? P->band_h[cls][q] : -1;
    if (rank) rank[q] = (conv && !P->rank_k[cls].empty()) ? P->rank_k[cls][q] : -1;
  }
  return CPC_OK;
}

int cpc_kernel_free(cpc_kernel* P) {
  if (!P) return CPC_OK;
  cudaFree(P->d_p);
  cudaFree(P->d_phat64);
  cudaFree(P->d_phat32);
  cudaFree(P->d_tw64);
  cudaFree(P->d_tw32);
  cudaFree(P->d_twp64);
  cudaFree(P->d_twp32);
  cudaFree(P->d_twp32_lo);
  cudaFree(P->d_hw32_lo);
  cudaFree(P->d_pp32);
  cudaFree(P->d_opf32);
  cudaFree(P->d_hw64);
  cudaFree(P->d_hw32);
  cudaFree(P->d_specw32);
  cudaFree(P->d_twdf);
  cudaFree(P->d_hwdf);
  cudaFree(P->d_phatdf);
  cudaFree(P->d_terms);
  cudaFree(P->d_taps32);
  cudaFree(P->d_taps64);
  cudaFree(P->d_cheb);
  cudaFree(P->d_tcheb32);
  cudaFree(P->d_tcheb64);
  cudaFree(P->d_lat);
  delete P;
  return CPC_OK;
}

}  // extern "C"

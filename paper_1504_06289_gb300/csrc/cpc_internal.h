// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <type_traits>

#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/cpc.h"

struct cpc_kernel {
  int n = 0;          // cells per axis
  double b = 0.0;     // half box edge
  double h = 0.0;     // 2b/n
  int M = 0;
  int R_N = 0;        // 2M+1
  int kind = 0;       // CPC_KERNEL_CONV / CPC_KERNEL_MASTER
  int len = 0;        // n (CONV) or 2n (MASTER)
  double hs = 0.0, u0 = 0.0;
  std::vector<double> t, a, p;  // host float64 tables, p is [R_N][len]

  // device tables
  double* d_p = nullptr;        // [R_N][len]
  // CONV only: spectrum of the length-2n even kernel, f = 0..n (real)
  double* d_phat64 = nullptr;   // [R_N][n+1]
  float* d_phat32 = nullptr;    // [R_N][n+1]
  // FFT tables for complex size n: tw[e] = exp(-2 pi i e / n), e < n;
  // half-angle table hw[f] = exp(-2 pi i f / (2n)), f <= n.
  double2* d_tw64 = nullptr;
  float2* d_tw32 = nullptr;
  double2* d_twp64 = nullptr;  // per-pass twiddle tables of the FFT plans (fft.cuh)
  float2* d_twp32 = nullptr;
  void* d_twp32_lo = nullptr;  // __half2: 2^24 (exact - float32) of each float32 pass-table entry
  void* d_hw32_lo = nullptr;   // the same for the half-angle table
  void* d_pp32 = nullptr;      // float2 [R_N][n]: kernel-term pairs (p^[f], p^[n-f])
  float4* d_opf32 = nullptr;   // [n]: float32 operand factors (1 + i e^{i theta_f}, 1 - i e^{i theta_f})
  double2* d_hw64 = nullptr;
  float2* d_hw32 = nullptr;
  // CONV only: Parseval weights d_q[2f+j] = w_f phat_q[f] / (2n), float32, [R_N][2(n+1)]
  float* d_specw32 = nullptr;
  // CONV only: how each kernel term is convolved (spectra.cu), per precision
  // class (0: float32 W, 1: float64 W): by the FFT, by the banded direct sum
  // (narrow terms, half-width H) or by the separable Chebyshev form (smooth
  // terms, rank K).  d_terms holds [class][kTermRows][R_N] ints: H per term
  // (-1: not banded), K per term (-1: not smooth), then the lists of banded,
  // smooth and FFT terms, of the terms contracted over the cells (banded then
  // FFT; the smooth terms' Gram matrices come from their moments), of the
  // lag-covered banded terms (H < n_lag: their Gram matrices are sums of the
  // n_lag lag Gram matrices) and the float32 energy path's contraction list
  // (banded terms with H >= n_lag, FFT terms, then n_lag entries whose W
  // slice slots, those of the first n_lag covered terms, hold the lag rows).  Banded taps p_q[0..kBandHalo] (float32 class: float2
  // (hi, lo); float64 class: double), zero beyond H; Chebyshev coefficients
  // C_q [R_N][16][16] float64 and the Chebyshev table T_k(x_i/b) [16][n]
  // (float2 (hi, lo) and double).
  int band_max[2] = {-1, -1};  // largest half-width sent to the banded kernel
  int rank_max[2] = {-1, -1};  // largest rank sent to the Chebyshev kernels
  int n_band[2] = {0, 0};
  int n_smooth[2] = {0, 0};
  int n_lag[2] = {0, 0};   // lag Gram matrices of the energy path (float32 class only)
  int n_cov[2] = {0, 0};   // banded terms they cover
  int n_eh[2] = {0, 0};    // entries of the energy path's contraction list
  std::vector<int> band_h[2];  // host copies of the half-widths and ranks
  std::vector<int> rank_k[2];
  // double-float copies (hi, lo) of the float64 FFT tables for the float64
  // forms other than CPC_FP64: pass twiddles [n] and half-angle factors
  // [n+1] as float4 (re hi, re lo, im hi, im lo), kernel spectra [R_N][n+1]
  // as float2
  float4* d_twdf = nullptr;
  float4* d_hwdf = nullptr;
  float2* d_phatdf = nullptr;
  int* d_terms = nullptr;
  float2* d_taps32 = nullptr;
  double* d_taps64 = nullptr;
  double* d_cheb = nullptr;
  float2* d_tcheb32 = nullptr;
  double* d_tcheb64 = nullptr;
  // MASTER kernels: scratch of the tensor-core sub-grid evaluation (the bf16
  // slices of the S3 rows, pre-swizzled per 64-point sub-tile, and their
  // exponents); calls on unordered streams sharing one kernel race on it
  unsigned char* d_lat = nullptr;
};

namespace cpc {

// where a convolution writes the tensor-core contraction's slices of W, in
// the chunk-blocked layout of its form: float32 W, three bf16 slices in
// 64-cell chunks [3][3 R_N][n/64][R_f][64]; float64 W (CPC_FP64_TC), five
// weighted bf16 slices in 32-cell chunks [5][3 R_N][n/32][R_f][32]; and the
// row exponents [3 R_f R_N] (row = col R_N + q)
struct SliceRows {
  __nv_bfloat16* out;
  long long slice_stride;  // elements between slices
  int* expo;
  int R_f;
};

// error reporting (thread-local message)
int fail(int status, const std::string& msg);

// optional CUDA-event timing of selected kernel launches (timing.cpp)
bool timing_on();
int timing_begin(const char* name, cudaStream_t s);  // -1 when not recording
void timing_end(int slot, cudaStream_t s);
int cuda_fail(cudaError_t e, const char* what);
void clear_error();

#define CPC_CUDA(call)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cpc::cuda_fail(e_, #call); \
  } while (0)

#define CPC_LAUNCH_CHECK(what)                                  \
  do {                                                          \
    cudaError_t e_ = cudaGetLastError();                        \
    if (e_ != cudaSuccess) return cpc::cuda_fail(e_, what);     \
  } while (0)

inline bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }
inline int ilog2(int n) { int l = 0; while ((1 << l) < n) ++l; return l; }
inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// host: sinc nodes and Galerkin vectors (newton_kernel.cpp)
void sinc_rule(int M, double h, double r_max, bool master, double* hs, double* u0);
double gauss_cell_integral(double t, double x0, double x1);
void build_twiddles(int n, std::vector<double>& tw_re, std::vector<double>& tw_im,
                    std::vector<double>& hw_re, std::vector<double>& hw_im);

// device-side builders (spectra.cu)
int build_pass_twiddles(cpc_kernel* P, cudaStream_t s);
size_t lattice_scratch_bytes(int n);
// nuclear factors F[l][a R_N + q][i] = p~_q[i - edges[l n_nuc + a]] of a MASTER
// kernel (edges: host int32 [3][n_nuc] in [0, n]), float64 or float32 (lattice.cu)
int launch_window(const cpc_kernel* P, int n_nuc, const int* edges, void* F, bool fp32, cudaStream_t s);
int compute_kernel_spectrum(cpc_kernel* P, cudaStream_t s);

// spectra of U columns into workspace (float64 and/or float32 copies)
int forward_spectra(const cpc_kernel* P, int ncols, const double* U, double2* Uhat64,
                    float2* Uhat32, cudaStream_t s);
// batched convolution from spectra.  U: the factor columns themselves
// (float64 [ncols][n]) or NULL; with U, the banded terms are convolved
// directly from U (band_conv_kernel), the smooth terms by the Chebyshev form
// (scratch: smooth_scratch_bytes, 256-byte aligned) and the FFT takes the rest
int convolve_from_spectra(const cpc_kernel* P, int ncols, const void* Uhat, void* W,
                          int precision, cudaStream_t s, const double* U = nullptr, void* scratch = nullptr);
// CPC_SPLIT and CPC_FP64_TC: the FFT terms in double-float arithmetic from
// double-float factor spectra (spectra_df_kernel), W in float64; banded and
// smooth terms as for CPC_FP64
int convolve_spectra_df(const cpc_kernel* P, int ncols, void* Uhat, double* W, cudaStream_t s, const double* U,
                        void* scratch, const SliceRows* so64 = nullptr);
bool conv_slices64_supported(const cpc_kernel* P);
// cp_convolve after argument checks; so64 (CPC_FP64_TC only, n >= 128): also
// write W's five-digit slices and row exponents for the contraction
int run_convolve(const cpc_kernel* P, int R_f, const double* U, void* W, int precision, void* ws, cudaStream_t s,
                 const SliceRows* so64 = nullptr);
int build_df_tables(cpc_kernel* P, cudaStream_t s);
// float32 convolution operands (X1, X2) from float64 transforms of U, and the
// convolutions from them (also writing the tensor-core contraction's W
// slices and row exponents, n >= 128, in the _sliced form); U as above
int forward_operands32(const cpc_kernel* P, int ncols, const double* U, void* X, cudaStream_t s);
size_t operands32_bytes(const cpc_kernel* P, int ncols);
int convolve_operands32(const cpc_kernel* P, int ncols, const void* X, float* W, cudaStream_t s,
                        const double* U = nullptr, void* scratch = nullptr);
int convolve_operands32_sliced(const cpc_kernel* P, int R_f, const void* X, float* W, __nv_bfloat16* slices,
                               long long slice_stride, int* expo, cudaStream_t s, const double* U = nullptr,
                               void* scratch = nullptr);
int build_kernel_pairs(cpc_kernel* P, cudaStream_t s);
// the convolution path of every kernel term, per precision class, from the
// host tables: banded if its half-width is at most band32 / band64, else
// Chebyshev if its rank is at most rank32 / rank64, else FFT (a negative
// maximum disables that path)
int build_term_tables(cpc_kernel* P, int band32, int band64, int rank32, int rank64, cudaStream_t s);
// the host part of build_term_tables (no device work): per class the ints
// [H per term][K per term][banded list][smooth list][FFT list], the taps, the
// Chebyshev coefficients [R_N][16][16] and the table T_k(x_i/b) [16][n]
constexpr int kTermRows = 8;  // rows of d_terms per precision class
constexpr int kMaxLags = 8;   // largest lag count of the tensor-core energy paths
struct TermPlan {
  std::vector<int> terms;  // [2][kTermRows][R_N]
  std::vector<float2> taps32;
  std::vector<double> taps64, cheb, tcheb;
  int n_band[2] = {0, 0}, n_smooth[2] = {0, 0}, n_lag[2] = {0, 0}, n_cov[2] = {0, 0}, n_eh[2] = {0, 0};
};
void plan_term_paths(const cpc_kernel* P, int band32, int band64, int rank32, int rank64, TermPlan& tp);
// default maxima: where the direct sum still costs less than the transform
// per output (float32 W: about 1.5 instructions per tap against about 110
// per output for the 8192-point float32 transform; float64 W: 2H + 1 float64
// operations against about 60); the Chebyshev form costs about 2K (float32)
// or K (float64) multiply-adds per output, below the transform for any K <= 16
constexpr int kDefaultBand32 = 20;
constexpr int kDefaultBand64 = 24;
constexpr int kDefaultRank = 16;
// scratch of the Chebyshev path (moments and coefficients of ncols columns)
size_t smooth_scratch_bytes(const cpc_kernel* P, int ncols);
// Gram matrices of the smooth terms from the moments and float64 coefficients
// that a convolution of the 3 R_f columns of U left in its scratch (spectra.cu):
// E_H partials (c given; cheb_gram_partials of them at most) and/or G
// [3][R_N][R_f][R_f] for those terms.  cheb_gram_active: the W type class has
// smooth terms (the convolution then takes them through the Chebyshev form
// whenever it is given U and its scratch); dense_terms: the others, which the
// cell contraction takes (n_q of them)
bool cheb_gram_active(const cpc_kernel* P, int cls);
const int* dense_terms(const cpc_kernel* P, int cls, int* n_q);
// the tensor-core energy path of W type class cls (FP32: 0, FP64_TC: 1): its
// contraction list (n_q entries, the last n_virtual of them lag rows; NULL:
// every term)
const int* eh_terms(const cpc_kernel* P, int cls, int* n_q, int* n_virtual);
// FP64_TC: the lag rows as five-digit float64 slices (as lag_slices32), and
// the covered terms' G = sum_m p_q[m] S_m in float64 into G [3][R_N][R_f][R_f]
int lag_slices64(const cpc_kernel* P, int R_f, const double* U, const SliceRows& so, cudaStream_t s);
int launch_lag_gram64(const cpc_kernel* P, int R_f, const double* S, double* G, cudaStream_t s);
// lag rows V_m = U shifted by +m plus U shifted by -m (V_0 = U), m < n_lag, as
// balanced three-digit slices with their row exponents in the W slice slots
// of the first n_lag covered terms (SliceRows of the float32 form)
int lag_slices32(const cpc_kernel* P, int R_f, const double* U, const SliceRows& so, cudaStream_t s);
// G and E_H partials of the covered terms from the lag Gram matrices S
// [3][n_lag][R_f][R_f]: G_q = sum_{m <= H_q} p_q[m] S_m
size_t lag_gram_partials(const cpc_kernel* P, int R_f);
int launch_lag_gram(const cpc_kernel* P, int R_f, const double* S, const double* c, double* G, double* partial,
                    long long* n_partial, cudaStream_t s);
size_t cheb_gram_partials(const cpc_kernel* P, int R_f);
int launch_cheb_gram(const cpc_kernel* P, int cls, int R_f, const void* scratch, const double* c, double* G,
                     double* partial, long long* n_partial, cudaStream_t s);
// rows-mode operands of the smooth terms (float32 W class, CONV kernel):
// Chebyshev moments of ncols float64 rows U [ncols][n] as float64 rows of
// `width` (k < 16, zeros beyond; Part: cheb_moment_rows_scratch bytes), and
// the coefficient rows d of the 3 R_rho columns a convolution left in its
// scratch, [3 R_rho n_smooth][width] float32 (row (l R_rho + m) n_smooth + j)
size_t cheb_moment_rows_scratch(const cpc_kernel* P, int ncols);
int cheb_moment_rows(const cpc_kernel* P, int ncols, const double* U, void* Part, double* out, int width,
                     cudaStream_t s);
int cheb_coef_rows(const cpc_kernel* P, int R_rho, const void* scratch, float* out, int width, cudaStream_t s);
// the convolution workspace without that scratch (which follows it)
size_t conv_spectra_bytes(const cpc_kernel* P, int R_f, int precision);

// float32 contractions (gram32.cu)
size_t eh32_partials(int R_f, int R_N);
int build_spectral_weights(const cpc_kernel* P, float* d, cudaStream_t s);
// (CPC_SPLIT, W64: qlist, when given, the n_q kernel terms to contract; the
// other terms' partial slots are zeroed)
int launch_eh32(const cpc_kernel* P, int R_f, const double* U, const float* W, const float* S32,
                const float* dtab, const double* c, double* G, double* partial, cudaStream_t s,
                const double* W64 = nullptr, const int* qlist = nullptr,
                int n_q = -1);
int launch_rows32(const cpc_kernel* P, int n_factors, const double* U_items, int N, const float* W,
                  const double* c_rho, double* rowpart, int groups, int tiles_per_cta, cudaStream_t s,
                  const double* W64 = nullptr);
size_t eh32a_partials(int R_f, int R_N);
size_t eh32a_u32_bytes(const cpc_kernel* P, int R_f);
int launch_eh32a(const cpc_kernel* P, int R_f, const double* U, const float* W, const double* c, double* G,
                 double* partial, float* U32, cudaStream_t s);
size_t tc_partials(int R_f, int R_N);
bool tc_supported(const cpc_kernel* P);
size_t tc_workspace(const cpc_kernel* P, int R_f);
int* tc_status_ptr(const cpc_kernel* P, int R_f, void* ws);
// CPC_FP64_TC: float64 operands in five bf16 slices, convolution matrices in float64
size_t tc64_partials(int R_f, int R_N);
size_t tc64_workspace(const cpc_kernel* P, int R_f);
int* tc64_status_ptr(const cpc_kernel* P, int R_f, void* ws);
// w_sliced: the convolution already wrote W's slices and row exponents where
// tc64_w_slices points; cheb_scratch: that convolution's scratch, whose
// moments give the smooth terms' G, the lag rows (lag_slices64, already in
// the W slices) the lag-covered terms' G (the cell contraction then takes
// only the other terms; NULL: every term by the cell contraction)
int launch_eh_tc64(const cpc_kernel* P, int R_f, const double* U, const double* W, const double* c, double* G,
                   double* partial, void* ws, cudaStream_t s, bool w_sliced = false,
                   const void* cheb_scratch = nullptr);
SliceRows tc64_w_slices(const cpc_kernel* P, int R_f, void* ws);
// tensor-core Coulomb-matrix rows (M item factors against Ns rho factors)
size_t tc_rows_workspace(const cpc_kernel* P, int M, int Ns);
size_t tc_rows_groups(const cpc_kernel* P, int Ns);
int* tc_rows_status_ptr(const cpc_kernel* P, int M, int Ns, void* ws);
// raster: 256-row blocks of item factors whose CTA pairs sweep the column tiles together;
// wmap: column s of the Ns is W row (s / n_wmap) R_N_src + wmap[s % n_wmap] (NULL: row s)
int launch_rows_tc(const cpc_kernel* P, int M, const double* U_items, int Ns, const float* W_rho,
                   const double* c_rho, double* rowpart, void* ws, cudaStream_t s, int raster,
                   const int* wmap = nullptr, int n_wmap = 1, int R_N_src = 1);
// where a convolution writes the W slices for launch_eh_tc(..., w_sliced = true)
void tc_w_slices(const cpc_kernel* P, int R_f, void* ws, __nv_bfloat16** slices, long long* slice_stride,
                 int** expo);
// qlist: the n_q kernel terms to contract (NULL: all); the partial slots of
// the others are zeroed; the last n_virtual entries are lag rows whose Gram
// matrices go to Gv [3][n_virtual][R_f][R_f]
int launch_eh_tc(const cpc_kernel* P, int R_f, const double* U, const float* W, const double* c, double* G,
                 double* partial, void* ws, cudaStream_t s, bool w_sliced = false, const int* qlist = nullptr,
                 int n_q = -1, double* Gv = nullptr, int n_virtual = 0);
// the V_H factors and spectra of CPC_SPLIT and CPC_FP64_TC are float64, like CPC_FP64
inline int storage_precision(int precision) { return precision == CPC_FP32 ? CPC_FP32 : CPC_FP64; }
inline bool known_precision(int precision) {
  return precision == CPC_FP64 || precision == CPC_FP32 || precision == CPC_SPLIT || precision == CPC_FP64_TC;
}
size_t spectra_bytes(const cpc_kernel* P, int ncols, int precision);

}  // namespace cpc

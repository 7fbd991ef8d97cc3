/*
 * cpc.h -- C ABI of the GB300 (sm_103a) rank-structured 3D Coulomb convolution.
 *
 * The library convolves functions given in canonical (CP) format on an
 * n x n x n cell-centred grid with the sinc-quadrature CP representation of
 * the Newton kernel 1/|x|, and forms the rank-sum contractions that give the
 * Hartree potential factors, the Hartree energy, Coulomb-matrix entries over
 * product functions and assembled lattice sums (Khoromskaia & Khoromskij,
 * arXiv:1504.06289: Sec. 2.5 Eqs. scal/had/conc/conv, Sec. 3.1, Sec. 3.2
 * Eq. Factor_Mk_Conv, Sec. 5.1 Eqs. refTensor/CoulombLatTensCan, Appendix 3
 * Eqs. galten/sinc_Newt/sinc_general).
 *
 * Conventions shared by every call
 *   Grid:   box [-b, b]^3, n cells per axis of width h = 2b/n, cell centres
 *           x_i = -b + (i + 1/2) h, i = 0..n-1.  n must be a power of two.
 *   CP data: side matrices are stored "column-major n x R" and the three
 *           axes are stacked, so a factor array for rank R is a contiguous
 *           [3][R][n] block: element (axis l, column k, cell i) lives at
 *           offset (l*R + k)*n + i.  Every column is n contiguous values.
 *   Pointers: unless marked "host", every pointer is DEVICE memory owned by
 *           the caller; the library never frees caller memory and, apart from
 *           make_newton_kernel's tables, never allocates.  Work that needs
 *           scratch takes a caller workspace (ws, ws_bytes) whose size comes
 *           from the matching *_workspace query; ws must be 256-byte aligned.
 *   Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy
 *           default stream).  Calls are stream-ordered and do not
 *           synchronise, except make_newton_kernel (which returns with its
 *           tables ready) and the host-side validation before any launch.
 *   Precision: CPC_FP64 computes in float64 throughout.  CPC_FP32 runs the
 *           bulk convolutions in float32 (V_H factors stored as float) and
 *           the contractions with float32 products, float32 partial sums over
 *           chunks of 256 cells and float64 cross-tile reductions.  CPC_SPLIT
 *           keeps the convolutions at float64 accuracy (V_H factors stored as
 *           double; the FFT terms in double-float arithmetic, pairs of
 *           float32 carrying about 48 bits, within about 1e-13 of CPC_FP64's
 *           float64 transform) and runs the contractions with float32
 *           products as in CPC_FP32, so E_H loses only the float32 rounding
 *           of its operands.  CPC_FP64_TC (cp_hartree_energy and
 *           cp_hartree_energy_from_factors only, n a multiple of 128) keeps
 *           the float64-accurate convolutions of CPC_SPLIT and runs the E_H contraction
 *           on the tensor cores: each float64 operand row is split exactly
 *           into five bf16 slices (40 bits of its row maximum), the slice
 *           pairs down to 2^-32 of the row scales are multiplied and summed
 *           exactly or below 2^-38 of the entry scale, and the convolution
 *           matrices and E_H are formed in float64 (the method's float64
 *           accuracy at tensor-core speed; every other entry point and the
 *           Coulomb, nuclear and lattice calls reject it with
 *           CPC_ERR_UNSUPPORTED and take CPC_FP64).  Kernel nodes, weights,
 *           cell integrals, spectra of the factors and final cross-rank
 *           reductions are float64 in every form.
 *   Errors: every entry point returns CPC_OK (0) or a negative status; no
 *           exception or abort crosses the ABI.  Arguments are validated on
 *           the host before any launch; a failed CUDA call returns
 *           CPC_ERR_CUDA and cpc_last_error() gives its message.
 */
#ifndef CPC_H
#define CPC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CPC_OK 0
#define CPC_ERR_INVALID -1      /* bad size, null pointer, inconsistent arguments */
#define CPC_ERR_WORKSPACE -2    /* workspace missing, misaligned or too small */
#define CPC_ERR_CUDA -3         /* a CUDA runtime call failed */
#define CPC_ERR_DEVICE -4       /* a device-side check flagged an error */
#define CPC_ERR_UNSUPPORTED -5  /* size or precision form not supported */

#define CPC_FP64 0
#define CPC_FP32 1
#define CPC_SPLIT 2
#define CPC_FP64_TC 3

#define CPC_KERNEL_CONV 0   /* cell-centred offsets m = -(n-1)..n-1 (Sec. 3.1) */
#define CPC_KERNEL_MASTER 1 /* 2n cells [jh,(j+1)h], j = -n..n-1 (Sec. 5.1, Eq. refTensor) */

typedef struct cpc_kernel cpc_kernel; /* opaque; owns device tables */

/* ---- a1/a2: the CP Newton kernel ------------------------------------------
 * make_newton_kernel -- Appendix 3, Eqs. sinc_Newt and galten; Sec. 5.1 Eq. refTensor.
 * Builds the R_N = 2M+1 term sinc quadrature 1/r ~ sum_q a_q exp(-t_q^2 r^2)
 * (nodes t_q = exp(u0 + k hs), a_q = 2 hs t_q / sqrt(pi), k = -M..M, with hs
 * and u0 balancing discretisation and truncation errors; all float64 on the
 * host) and the Galerkin vectors p_q = a_q^{1/3} * (cell integrals of
 * exp(-t_q^2 x^2)).  kind = CPC_KERNEL_CONV stores p_q[m], m = 0..n-1 (the
 * vector is even in m) and its length-2n real spectrum for FFT convolution;
 * CPC_KERNEL_MASTER stores p~_q[j], j = -n..n-1 (column j+n).
 * n: power of two, 16 <= n <= 16384 (CONV: n <= 8192).  b > 0.  1 <= M <= 64.
 * Allocates device memory for its tables (released by cpc_kernel_free) and
 * synchronises the given stream before returning.  *out receives the handle. */
int make_newton_kernel(int n, double b, int M, int kind, void* stream, cpc_kernel** out);

/* The float64 host part of make_newton_kernel alone, with no device work:
 * t[R_N], a[R_N], p[R_N][len] (len = n for CONV, 2n for MASTER), and the
 * step hs and shift u0 of the quadrature, into caller HOST buffers (any
 * pointer may be NULL).  Same argument rules as make_newton_kernel. */
int make_newton_kernel_tables(int n, double b, int M, int kind, double* t, double* a, double* p,
                              double* hs, double* u0);

/* Scalars of a kernel (any pointer may be NULL). */
int cpc_kernel_info(const cpc_kernel* P, int* n, double* b, int* M, int* R_N, int* kind,
                    double* hs, double* u0);

/* Host copies of the float64 tables: t[R_N], a[R_N] and p[R_N][len] with
 * len = n (CONV) or 2n (MASTER).  Any pointer may be NULL.  host pointers. */
int cpc_kernel_tables(const cpc_kernel* P, double* t, double* a, double* p);

/* Releases the kernel's device tables and the handle (NULL is a no-op). */
int cpc_kernel_free(cpc_kernel* P);

/* How each kernel term of a CONV kernel is convolved (Sec. 2.5, Eq. conv)
 * by cp_convolve and every call that convolves U; all three give W = p_q * U
 * to within the rounding of the W type:
 *  - banded: the Galerkin vector of a term with a large exponent t_q is a few
 *    cells wide; W is the direct sum over |m| <= H_q, H_q the smallest
 *    half-width whose tail 2 sum_{m > H_q} |p_q[m]| is at most 2^-32 (float32
 *    W) or 2^-60 (float64 W) of |p_q[0]| + 2 sum_{m>0} |p_q[m]|, rounded up
 *    to an instantiated width (0..8, 10..16 step 2, 20..32 step 4);
 *  - smooth: a term with a small exponent is, on [-b, b]^2, the polynomial
 *    p_q(x - y) ~ sum_{k,l<K} C_kl T_k(x/b) T_l(y/b) (Chebyshev, K in
 *    {4, 8, 12, 16}, within 2^-34 (float32 W) or 2^-46 (float64 W) of p_q[0]
 *    on a lattice of grid cells); W = sum_k d_k T_k(x_i/b) with
 *    d = C (sum_j T_l(x_j/b) U[j]);
 *  - FFT: every other term (length-2n real transforms).
 * make_newton_kernel sets the largest half-width to 20 (float32 W) and 24
 * (float64 W) and the largest rank to 16.  cpc_kernel_set_conv_paths sets
 * them (half-widths in [-1, 32], ranks in [-1, 16]; -1 disables that path),
 * rebuilds the device tables on `stream` and synchronises it; no call that
 * uses P may run meanwhile.  cpc_kernel_conv_paths writes, for the W type of
 * `precision`, each term's half-width (or -1) into half_width[R_N] and rank
 * (or -1) into rank[R_N], host arrays, either may be NULL.
 * cp_convolve_from_spectra has no U and takes the FFT for every term. */
int cpc_kernel_set_conv_paths(cpc_kernel* P, int max_half_width32, int max_half_width64, int max_rank32,
                              int max_rank64, void* stream);
int cpc_kernel_conv_paths(const cpc_kernel* P, int precision, int* half_width, int* rank);

/* The host part of the path choice alone, with no device work (CONV kernel
 * of make_newton_kernel(n, b, M), limits as cpc_kernel_set_conv_paths):
 * half_width[2][R_N] and rank[2][R_N] (row 0: float32 W, row 1: float64 W;
 * -1 where the path is not taken) and the Chebyshev coefficients
 * cheb[R_N][16][16] (C_q[k][l]; zero for terms never fitted), all HOST
 * arrays, any may be NULL. */
int make_newton_kernel_paths(int n, double b, int M, int max_half_width32, int max_half_width64, int max_rank32,
                             int max_rank64, int* half_width, int* rank, double* cheb);

/* The energy paths' contraction plan of the same kernel, host only:
 * plan[2][3] (HOST array; row 0: float32 W, row 1: float64 W) = the number
 * L of lag Gram matrices S_m = U^T (U shifted by +m plus U shifted by -m),
 * m < L (L minimises L plus the number of banded terms with half-width
 * >= L, at most 8, with at least L terms below it), the number of banded
 * terms with half-width < L whose convolution matrices are the sums
 * sum_{m <= H} p_q[m] S_m (Sec. 3.2 Eq. Factor_Mk_Conv with the banded sum
 * of Sec. 2.5 Eq. conv), and the number of rows the tensor-core contraction
 * takes over the cells (banded terms with half-width >= L, FFT terms, L lag
 * rows; the smooth terms' matrices come from their Chebyshev moments).  The
 * FP32 and FP64_TC energy paths (cp_hartree_energy) use rows 0 and 1. */
int make_newton_kernel_eh_plan(int n, double b, int M, int max_half_width32, int max_half_width64, int max_rank32,
                               int max_rank64, int* plan);

/* ---- a3: grid sampling of Gaussians (Sec. 3.1, Eq. disc_GTO) --------------
 * U[l][k][i] = exp(-a_k (x_i - X[k][l])^2) for R Gaussians exp(-a_k |x - X_k|^2).
 * a: [R], X: [R][3] (row k holds X_k), U: [3][R][n]; all float64 device. */
int cp_sample_gaussians(int n, double b, int R, const double* a, const double* X, double* U,
                        void* stream);

/* ---- A2: Hadamard products of factor pairs (Sec. 2.5, Eq. had) ------------
 * For r = 0..n_pairs-1 and every axis l:
 *   out[l][r][:] = F[l][pa[r]][:] * F[l][pb[r]][:]   (elementwise),
 *   c_out[r]     = scale[r] * d[pa[r]] * d[pb[r]]      (scale may be NULL = 1).
 * F: [3][n_in][n] float64; pa, pb: [n_pairs] int32 in [0, n_in); d: [n_in];
 * out: [3][n_pairs][n]; c_out: [n_pairs].  Builds the CP factors of product
 * functions g_mu g_nu and of densities from sampled primitives. */
int cp_hadamard_pairs(int n, int n_in, int n_pairs, const int* pa, const int* pb,
                      const double* F, const double* d, const double* scale,
                      double* out, double* c_out, void* stream);

/* ---- a4: batched 1D convolutions (Sec. 2.5 Eq. conv; V_H of Sec. 3.1) -----
 * W[l][k*R_N + q][i] = sum_{j=0}^{n-1} U[l][k][j] * p_q[i - j],  i = 0..n-1,
 * for every axis l, rank k < R_f and kernel term q < R_N of a CONV kernel:
 * the factors of V_H = f * P_R.  U: [3][R_f][n] float64.  W: [3][R_f*R_N][n],
 * float64 for CPC_FP64, CPC_SPLIT and CPC_FP64_TC, float32 for CPC_FP32
 * (CPC_SPLIT and CPC_FP64_TC: the FFT terms in double-float arithmetic,
 * within about 1e-13 of CPC_FP64).  Implemented as length-2n real
 * FFT convolutions in the chosen precision (the spectra of U are formed in
 * float64), except for the narrow kernel terms, summed directly over their
 * band, and the smooth ones, evaluated in their separable Chebyshev form
 * (cpc_kernel_set_conv_paths).  Workspace: cp_convolve_workspace bytes. */
size_t cp_convolve_workspace(const cpc_kernel* P, int R_f, int precision);
int cp_convolve(const cpc_kernel* P, int R_f, const double* U, void* W, int precision,
                void* ws, size_t ws_bytes, void* stream);

/* The two halves of cp_convolve with the factor spectra as an explicit,
 * caller-owned intermediate.  spec: [3][R_f][n+1] complex bins of the
 * zero-padded length-2n columns, interleaved (re, im), float64 (CPC_FP64) or
 * float32 (CPC_FP32: computed in float64, rounded once).  16-byte aligned. */
int cp_factor_spectra(const cpc_kernel* P, int R_f, const double* U, void* spec, int precision,
                      void* stream);
int cp_convolve_from_spectra(const cpc_kernel* P, int R_f, const void* spec, void* W, int precision,
                             void* stream);

/* ---- a5/a6: convolution matrices and the Hartree energy -------------------
 * G[l][q][k'][k] = sum_i U[l][k'][i] W[l][k*R_N+q][i]   (Sec. 3.2,
 *                  Eq. Factor_Mk_Conv: U^T (p_q * U), symmetric in k', k),
 * E_H = h^3 sum_q sum_{k,k'} c_k c_k' prod_l G[l][q][k'][k]
 *     = h^3 <f, P_R * f>      (Sec. 2.5 Eq. scal with Eq. conv).
 * Runs cp_convolve into W (required: it receives the V_H factors, type as
 * in cp_convolve), then the contraction of U with W: float64 throughout for
 * CPC_FP64.  CPC_FP32 (n a multiple of 128): on the tensor cores, each row
 * of U and of the float32 W split exactly into three bf16 integer slices under
 * a per-row power-of-two scale (the convolution writes W's slices in the same
 * pass as W), the slice products summed in TMEM over 512-cell groups (all
 * three slice groups exactly, W in balanced digits)
 * and folded into a compensated float32 sum per entry (at least as accurate
 * as float32 operands with float32 products); other n: float32 products on
 * CUDA cores.  CPC_SPLIT: float32
 * products of U and W (rounded on load), compensated float32 accumulation.
 * CPC_FP64_TC: five weighted bf16 slices per float64 operand on the tensor
 * cores, G in float64.  The same G by other orders of the same sums, in the
 * CPC_FP32, CPC_SPLIT and CPC_FP64_TC forms: a smooth term's (Chebyshev path)
 * from its moments, G[k'][k] = sum_j m_k'[j] d_k[j] with d_k = C_q m_k
 * (double-float sums), and in CPC_FP32 and CPC_FP64_TC a narrow term's
 * (banded path, half-width H below the plan's lag count L) from lag Gram
 * matrices, G = sum_{m <= H} p_q[m] U^T (U shifted by +m plus U shifted by
 * -m) (make_newton_kernel_eh_plan); the other terms are contracted over the
 * cells.  CPC_FP64 contracts every term over the cells.
 * All forms reduce across tiles in float64.  If a device-side wait of the
 * tensor-core kernel gives up, E_H is written as NaN.  c: [R_f] float64.  G: NULL or
 * [3][R_N][R_f][R_f] float64 (needed by the adjoint).  E_H: one float64 on
 * the device.  Workspace: cp_hartree_energy_workspace bytes. */
size_t cp_hartree_energy_workspace(const cpc_kernel* P, int R_f, int precision);
int cp_hartree_energy(const cpc_kernel* P, int R_f, const double* U, const double* c, void* W,
                      double* G, double* E_H, int precision, void* ws, size_t ws_bytes,
                      void* stream);

/* The contraction part of cp_hartree_energy alone: G and E_H from existing
 * V_H factors W (as written by cp_convolve with the same precision), in the
 * spatial form (float32 products on the float32 factors for CPC_FP32).
 * Workspace: cp_hartree_energy_from_factors_workspace bytes. */
size_t cp_hartree_energy_from_factors_workspace(const cpc_kernel* P, int R_f, int precision);
int cp_hartree_energy_from_factors(const cpc_kernel* P, int R_f, const double* U, const double* c,
                                   const void* W, double* G, double* E_H, int precision, void* ws,
                                   size_t ws_bytes, void* stream);

/* E_H without the V_H factors: the convolution matrices by Parseval on the
 * length-2n circle from float32 spectra (as written by cp_factor_spectra
 * with CPC_FP32), G_q[k',k] = (1/2n) sum_f w_f p^_q[f] Re(U^_k'[f] conj U^_k[f]),
 * w_0 = w_n = 1, else 2; float32 products and sums (chunks of 256), float64
 * final reduction.  G (may be NULL) and E_H as in cp_hartree_energy.  The
 * spectral sums cancel, so the error is comparable to the spatial float32
 * form at twice its flops; it needs no V_H factors.  precision: CPC_FP32.
 * Workspace: cp_hartree_energy_from_spectra_workspace bytes. */
size_t cp_hartree_energy_from_spectra_workspace(const cpc_kernel* P, int R_f);
int cp_hartree_energy_from_spectra(const cpc_kernel* P, int R_f, const void* spec, const double* c,
                                   double* G, double* E_H, int precision, void* ws, size_t ws_bytes,
                                   void* stream);

/* cp_hartree_energy without a workspace argument, for callers that cannot
 * allocate device memory (a host program that owns a fixed device pool from
 * start-up, a plug-in living inside another runtime's allocator, a real-time
 * loop where cudaMalloc's synchronisation and latency are not allowed).  The
 * paper has no counterpart: this is a packaging variant of the same
 * computation, with the same arguments as cp_hartree_energy minus ws.
 * Its scratch is one file-scope device array of 32 MiB, held by every GPU
 * that loads the library until the process exits; a call needs
 * cp_hartree_energy_workspace(P, R_f, precision) bytes of it.
 * Sizes whose requirement exceeds 32 MiB are rejected with
 * CPC_ERR_UNSUPPORTED and a message naming both sizes; nothing is launched.
 * A device address of the array is valid only in the CUDA context it was
 * looked up in, so every call that is not under stream capture looks it up in
 * the current context (keyed by context: a caller's own non-primary context,
 * or a primary context recreated after cudaDeviceReset, gets its own); under
 * capture the address from an earlier call in the same context is used, so
 * make the first call in a context before any stream capture (otherwise
 * CPC_ERR_INVALID).  Invalid arguments are reported as CPC_ERR_INVALID before
 * the size limit is applied.  Every call on a device shares the array and sees the last
 * call's bytes there; the kernels overwrite all scratch they read, so no
 * clearing is needed, but calls whose work overlaps on the GPU (unordered
 * streams) race on it.  No cudaMalloc, cudaFree or allocating library call
 * is made. */
int cp_hartree_energy_noalloc(const cpc_kernel* P, int R_f, const double* U, const double* c, void* W,
                              double* G, double* E_H, int precision, void* stream);

/* ---- a7: adjoint of E_H ---------------------------------------------------
 * Derived from Sec. 2.5 Eq. scal and Eq. conv (each Toeplitz factor of p_q is
 * symmetric):
 *   dU[l][m][:] = 2 h^3 c_m sum_q sum_k' c_k' H_q^l[m][k'] W[l][k'*R_N+q][:],
 *   H_q^l = prod_{l' != l} G[l'][q]  (elementwise),
 *   dc[m]       = 2 h^3 sum_q sum_k' c_k' prod_l G[l][q][m][k'].
 * W and G as produced by cp_hartree_energy with the same precision.
 * dU: [3][R_f][n] float64, dc: [R_f] float64 (dc may be NULL). */
int cp_hartree_energy_adjoint(const cpc_kernel* P, int R_f, const double* c, const void* W,
                              const double* G, double* dU, double* dc, int precision,
                              void* stream);

/* Chain rule from dU to the Gaussians of cp_sample_gaussians:
 *   da[k]    = sum_l sum_i dU[l][k][i] * (-(x_i - X_kl)^2) * U[l][k][i],
 *   dX[k][l] = sum_i dU[l][k][i] * 2 a_k (x_i - X_kl) * U[l][k][i].
 * a [R], X [R][3], U, dU [3][R][n]; da [R], dX [R][3]; float64 device. */
int cp_gaussian_param_grad(int n, double b, int R, const double* a, const double* X,
                           const double* U, const double* dU, double* da, double* dX,
                           void* stream);

/* ---- a8: Coulomb matrix over product functions (Sec. 3.1, J_km) ----------
 * For item t with CP factors u_r, r in [off[t], off[t+1]) (coefficients c_items[r])
 * and the density rho = sum_m c_rho[m] u_m^(1) (x) u_m^(2) (x) u_m^(3):
 *   J[t] = h^3 sum_r c_items[r] sum_m c_rho[m] sum_q prod_l <u_r^(l), W_rho[l][m*R_N+q]>,
 * with W_rho = the V_H factors of rho (computed here into W_rho, type as in
 * cp_convolve).  off: [n_items+1] int32 device, nondecreasing, off[0] = 0 and
 * off[n_items] = n_factors (the caller's contract: offsets outside
 * [0, n_factors] are clamped, never dereferenced); U_items: [3][n_factors][n];
 * c_items: [n_factors]; U_rho: [3][R_rho][n]; c_rho: [R_rho]; J: [n_items]
 * float64.  Item factors are concatenated into one row space, so items of
 * uneven rank share tiles and no item leaves a tile idle.  CPC_FP64, CPC_SPLIT
 * (and CPC_FP32 when n is not a multiple of 128): one persistent launch over
 * (row tile, column group) work units, a column group being tiles_per_cta
 * consecutive 64-column tiles of the R_rho*R_N V_H columns.  CPC_FP32 with n
 * a multiple of 128: the tensor-core contraction of cp_hartree_energy (exact
 * bf16 slices of the item factors and of the float32 W_rho) with the
 * R_rho R_N columns (m, q) taken as one-term factors, on tiles of 256 item
 * factors x 128 columns; tiles_per_cta is then the number of 256-row item
 * blocks whose CTA pairs sweep the column tiles together (a raster group:
 * the pairs in flight share row blocks and column tiles in L2; capped at
 * the number of blocks).  tiles_per_cta: 0 = default 8, else a power of two
 * in [1, 128].  The result does not depend on it (fixed-order reductions).
 * If one of the tensor-core form's device-side waits gives up, J is written
 * as NaN.  Stream-ordered and allocation-free, so
 * a sequence of these calls can be captured in a CUDA graph.  Workspace:
 * coulomb_matrix_workspace bytes (sized for the smallest tiles_per_cta; for
 * the tensor-core form it holds the bf16 slices, 18 n (n_factors + R_rho R_N)
 * bytes). */
size_t coulomb_matrix_workspace(const cpc_kernel* P, int n_items, int n_factors, int R_rho,
                                int precision);
int coulomb_matrix(const cpc_kernel* P, int n_items, const int* off, int n_factors, const double* U_items,
                   const double* c_items, int R_rho, const double* U_rho, const double* c_rho,
                   void* W_rho, double* J, int precision, int tiles_per_cta, void* ws, size_t ws_bytes,
                   void* stream);

/* Galerkin matrix of the nuclear potential over product functions (Sec. 3.3):
 * the reference Newton kernel of a MASTER kernel shifted onto each nucleus
 * by the rank-1 windowing operator,
 *   F[l][a R_N + q][i] = p~_q[i - nuc_edges[l][a]],  i = 0..n-1
 * (computed here into F), gives P_c = sum_a Z[a] sum_q prod_l F[l][a R_N + q]
 * (h^3 times V_c = -sum Z_a / |x - a_a| at the cell centres, up to the sign),
 * and
 *   V[t] = -sum_{r in item t} c_items[r] sum_a Z[a] sum_q prod_l <u_r^(l), F[l][a R_N + q]>
 * = -<G_k . G_m, P_c> for item t = (k, m) given as the CP factors of
 * G_k . G_m (as in coulomb_matrix).  A nucleus sits at the grid-cell edge
 * nuc_edges[l][a] of each axis (x = -b + e h).  off, U_items, c_items: as in
 * coulomb_matrix; n_nuc in [1, 256] with n_nuc R_N <= 65535; nuc_edges: host
 * int32 [3][n_nuc] in [0, n]; Z: device float64 [n_nuc]; F: [3][n_nuc R_N][n]
 * float64 (CPC_FP64, CPC_SPLIT) or float32 (CPC_FP32); V: device float64
 * [n_items].  The contraction is coulomb_matrix's for each form over the
 * n_nuc R_N columns (a, q), the product over axes being per column (the
 * tensor-core form for CPC_FP32 with n a multiple of 128; a device-side wait
 * that gives up writes NaN).  Workspace: nuclear_matrix_workspace bytes,
 * 256-byte aligned.  Returns CPC_OK, CPC_ERR_INVALID (not a MASTER kernel,
 * NULL or misaligned pointer, edge out of range), CPC_ERR_UNSUPPORTED,
 * CPC_ERR_WORKSPACE or CPC_ERR_CUDA; no launch happens on an argument error. */
size_t nuclear_matrix_workspace(const cpc_kernel* master, int n_items, int n_factors, int n_nuc, int precision);
int nuclear_matrix(const cpc_kernel* master, int n_items, const int* off, int n_factors, const double* U_items,
                   const double* c_items, int n_nuc, const int* nuc_edges, const double* Z, void* F, double* V,
                   int precision, void* ws, size_t ws_bytes, void* stream);

/* Schedule tuner for coulomb_matrix: computes W_rho, then times the
 * contraction for every candidate schedule on the caller's data (one untimed
 * and one timed launch each, CUDA events on `stream`; this call synchronises
 * the stream), writes the fastest to *best_tiles_per_cta (and its time in ms
 * to *best_ms if not NULL) and leaves J computed with it.  Candidates:
 * tiles_per_cta in {4, 8, ..., 128} for the CUDA-core forms, raster groups
 * {1, 2, 4, ..., 32} for the tensor-core form.  times_ms (NULL, or host
 * float[8]): times_ms[k] = the timed launch of candidate 2^k, NaN where 2^k
 * is not a candidate.  Same arguments as coulomb_matrix otherwise. */
int coulomb_matrix_tune(const cpc_kernel* P, int n_items, const int* off, int n_factors,
                        const double* U_items, const double* c_items, int R_rho, const double* U_rho,
                        const double* c_rho, void* W_rho, double* J, int precision, void* ws,
                        size_t ws_bytes, void* stream, int* best_tiles_per_cta, float* best_ms,
                        float* times_ms);

/* ---- two-electron integrals: 1D density fitting + truncated Cholesky (Sec. 3.2) ----
 * For N_b s-type primitive Gaussians with sampled factors U_prims [3][n_b][n]
 * (device float64, cp_sample_gaussians) and n_pairs pairs P = (pa[P], pb[P])
 * (device int32, entries in [0, n_b)), the side matrices
 * G^(l)[i, P] = U_prims[l][pa[P]][i] U_prims[l][pb[P]][i] are fitted per axis
 * (Eq. 1DDensFit) by a truncated Cholesky factorisation with diagonal
 * pivoting of G G^T, stopped when the largest remaining diagonal is
 * <= tol_df times the largest initial one or after max_rank_df (<= 128)
 * steps: G ~ U V^T with U = L L[I,:]^{-1} and V = G[I,:]^T (I the pivots).
 * With M_k^(l) = U^(l)T (p_k * U^(l)) (Eq. Factor_Mk_Conv; P a CONV kernel),
 * the TEI matrix b_{P,P'} = <G_P, P_R * G_P'> (Eq. TEI_tens) is
 *   B = h^3 sum_k (Hadamard over l) V^(l) M_k^(l) V^(l)T,
 * whose diagonal and pivot columns drive the same truncated Cholesky
 * factorisation (tol_b, max_rank_b <= n_pairs): B ~ L L^T.  Output: L
 * [max_rank_b][n_pairs] device float64 (column s of L at L + s n_pairs, zero
 * beyond the rank) and ranks device int32[4] = (R_1, R_2, R_3, R_B).  The
 * pivot loops run on the device (no host synchronisation); float64
 * throughout.  Workspace: tei_cholesky_workspace bytes, 256-byte aligned.
 * Returns CPC_OK, CPC_ERR_INVALID (not a CONV kernel, bad pointer or size,
 * negative tolerance), CPC_ERR_UNSUPPORTED (max_rank_df > 128),
 * CPC_ERR_WORKSPACE or CPC_ERR_CUDA. */
size_t tei_cholesky_workspace(const cpc_kernel* P, int n_pairs, int max_rank_b);
int tei_cholesky(const cpc_kernel* P, int n_b, const double* U_prims, int n_pairs, const int* pa, const int* pb,
                 double tol_df, double tol_b, int max_rank_df, int max_rank_b, double* L, int* ranks, void* ws,
                 size_t ws_bytes, void* stream);

/* Coulomb matrix of a density matrix D (device float64 [n_b][n_b],
 * symmetric) from the TEI factor of tei_cholesky (Sec. 3.2):
 *   J[P] = sum_{P'} b_{P,P'} (2 - delta_{pa pb}) D[pa[P']][pb[P']]  ~  (L (L^T d))[P]
 * for every pair P (J: device float64 [n_pairs]; with all pairs mu <= nu,
 * J[P] = J_{pa[P] pb[P]}).  L, ranks: as written by tei_cholesky.  Workspace:
 * 256-byte aligned, at least align256(8 n_pairs) + 8 max_rank_b bytes.
 * Returns CPC_OK, CPC_ERR_INVALID, CPC_ERR_WORKSPACE or CPC_ERR_CUDA. */
int tei_coulomb(int n_b, int n_pairs, const int* pa, const int* pb, int max_rank_b, const double* L,
                const int* ranks, const double* D, double* J, void* ws, size_t ws_bytes, void* stream);

/* Exchange matrix of a density matrix D from the TEI factor (Sec. 3.1, the
 * exchange operator K_km,a = <G_k . phi_a, (G_m . phi_a) * P_R> summed over the
 * orbitals phi_a = sum_mu c_{mu a} g_mu, D = sum_a c_a c_a^T):
 *   K[k][m] = sum_{mu,nu} D[mu][nu] b_{(k mu),(m nu)}  ~  sum_{s < R_B} (X_s D X_s^T)[k][m],
 *   X_s[k][mu] = L[s][pair of g_k g_mu]
 * (a product g_k g_mu with no pair in (pa, pb) contributes 0).  n_b <= 1024;
 * D, K: device float64 [n_b][n_b]; L, ranks as written by tei_cholesky.
 * Workspace: tei_exchange_workspace(n_b, max_rank_b) bytes, 256-byte
 * aligned.  Returns CPC_OK, CPC_ERR_INVALID, CPC_ERR_WORKSPACE or CPC_ERR_CUDA. */
size_t tei_exchange_workspace(int n_b, int max_rank_b);
int tei_exchange(int n_b, int n_pairs, const int* pa, const int* pb, int max_rank_b, const double* L,
                 const int* ranks, const double* D, double* K, void* ws, size_t ws_bytes, void* stream);

/* ---- a9/a10: assembled lattice sums (Sec. 5.1, Eq. CoulombLatTensCan) -----
 * With a MASTER kernel p~_q and, per axis l, L[l] charge positions given as
 * grid-cell edge indices e[l][k] in [0, n] (a charge at x = -b + e h):
 *   S[l][q][i] = sum_{k < L[l]} p~_q[i - e[l][k]],  i = 0..n-1     (a9)
 * and, when V is not NULL, the potential on the tensor sub-grid
 *   V[s1][s2][s3] = h^-3 sum_q S[1][q][sub[0][s1]] S[2][q][sub[1][s2]] S[3][q][sub[2][s3]]
 * for s_l < n_sub (a10; row-major, s3 fastest).  L: host int32[3], each in
 * [0, 256]; edges: host int32 array of L[0]+L[1]+L[2] entries (axis 0
 * first), each in [0, n]; sub: device int32 [3][n_sub] in [0, n) (entries
 * outside are clamped), 1 <= n_sub <= 512.  R_N <= 129.
 * S: [3][R_N][n] float64.  V: n_sub^3 float64 (CPC_FP64) or float32
 * (CPC_FP32: for R_N <= 64 on the tensor cores, the pair products S1 S2 and
 * S3 rounded to float32, each row of them split exactly into four bf16
 * integer slices under a per-row power of two, slice products summed exactly
 * in TMEM and folded into float32 once per value; a device-side wait that
 * gives up writes NaN; for R_N > 64 float32 products with a float32
 * compensated sum). */
int lattice_potential_sum(const cpc_kernel* master, const int* L, const int* edges, double* S,
                          int n_sub, const int* sub, void* V, int precision, void* stream);

/* Interaction energy of equal charges Z on the tensor lattice of grid-cell
 * edges (Sec. 5.3): the sum E_L = 1/2 sum_{k != j} Z^2 / |x_k - x_j|
 * (Eq. EnergyLatSum) as the rank-R_N lattice sum traced at the lattice points
 * with the singular-point correction (Eq. EnergyLattice):
 *   E_L = Z^2 h^-3 / 2 sum_q (prod_l T_q^(l) - L[0] L[1] L[2] t0_q^3),
 *   T_q^(l) = 1/2 sum_{j,k < L[l]} (p~_q[e_j - e_k - 1] + p~_q[e_j - e_k]),
 *   t0_q = (p~_q[-1] + p~_q[0]) / 2,
 * in float64 (the pairs of each axis counted once per difference d = e_j - e_k,
 * then O(R_N) work per distinct d): a charge at edge e is the corner shared by the
 * cells e-1 and e of each axis, and the tensor value at a lattice point is
 * read as the mean over those 8 cells (a cube of edge 2h centred on the point,
 * whose mean of the harmonic 1/r has no second-order error).  Accurate when
 * the charges are many cells apart (about 30 or more).  master: a MASTER
 * kernel; L: host int32[3], each in [0, 256]; edges: host int32 array of
 * L[0]+L[1]+L[2] entries (axis 0 first), each in [1, n-1]; Z finite; E_L:
 * device float64, written once.  Uses the kernel's scratch (calls on
 * unordered streams sharing one kernel race on it).  Returns CPC_OK,
 * CPC_ERR_INVALID (not a MASTER kernel, NULL argument, edge out of range,
 * Z not finite), CPC_ERR_UNSUPPORTED (L out of range) or CPC_ERR_CUDA; no
 * launch happens on an error. */
int lattice_interaction_energy(const cpc_kernel* master, const int* L, const int* edges, double Z,
                               double* E_L, void* stream);

/* ---- status -------------------------------------------------------------- */
/* ---- kernel timing (measurement support; the paper has no counterpart) -----
 * While enabled, every launch of spectra_kernel, conv_kernel,
 * slice_rows_kernel, gemm3_tc_kernel, subgrid_tc_kernel, lattice_pairs_kernel,
 * lattice_energy_kernel and adjoint_gemm_kernel, and each phase of
 * tei_cholesky (tei_fit, tei_conv_matrices, tei_factor), is bracketed by two CUDA events recorded on the stream the
 * kernel is launched on (up to 8192 launches; later ones go unrecorded).
 * cpc_kernel_timing(1) creates the events on first use and clears earlier
 * records; cpc_kernel_timing(0) stops recording and keeps the records.
 * cpc_kernel_timing_read(name, total_ms, launches) waits for the recorded
 * events of that kernel name and returns their summed device time (ms) and
 * count (0 and 0 for an unknown name).  Host-side only; not for use inside a
 * stream capture.  Returns CPC_OK, CPC_ERR_INVALID (null argument) or
 * CPC_ERR_CUDA. */
int cpc_kernel_timing(int enable);
int cpc_kernel_timing_read(const char* kernel, double* total_ms, int* launches);

const char* cpc_status_string(int status);
/* Message of the most recent failure in this thread ("" if none). */
const char* cpc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CPC_H */

/*
 * helicwave.h -- C ABI of the GB300 (sm_103a) library for the helical-wave spectral method
 * (Agarwal & Banerjee, arXiv 2210.12252): matrix-free Hamiltonian x block products, the
 * diagonal preconditioner and a block eigensolver, for many (eta, nu) points.
 *
 * Conventions for every call
 *   - Units: Hartree and bohr.
 *   - Complex arrays are interleaved (re, im) FP64 pairs ("complex128"), column-major with a
 *     leading dimension ld >= L_k counted in complex entries: entry (i, j) is at
 *     ptr[2*(i + j*ld)] (real) and ptr[2*(i + j*ld) + 1] (imag).
 *   - Device pointers are caller-owned device memory on the context's device; the library
 *     never frees them.  The library owns its tables and workspace, sized by hw_setup_basis;
 *     hw_apply_H / hw_apply_precond allocate nothing.
 *   - Calls are ordered on the context's CUDA stream and asynchronous unless stated
 *     (hw_solve_eigs, the hw_get_* queries and hw_build_potential return with results on the
 *     host).  A context is not thread-safe.
 *   - Errors: every call returns an hw_status; nothing throws across the ABI.  The message of
 *     the last failure is hw_last_error(ctx).  Invalid arguments are rejected on the host
 *     before any launch (HW_EINVAL); device-side waits are bounded and report HW_ETIMEOUT.
 *
 * Reciprocal-space order (compact): the order of eq. wavefun_storage,
 *     i(m,n,k) = (m+M)(2N+1)K + (n+N)K + k,
 * restricted to the modes kept by the kinetic-energy cutoff of eq. Energy_cutoff at the
 * k-point (mask of Sec. "Imposition of kinetic energy cutoff").  L_k is the kept count.
 * Real-space order: eq. wavefun_storage_real, theta1 slowest, r fastest, with theta1_i =
 * i/N_th1, theta2_j = j/(Ncyc N_th2) and r_p the Gauss-Jacobi(0,1) nodes on (0, R) in
 * ascending order.
 */
#ifndef HELICWAVE_H
#define HELICWAVE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hw_ctx hw_ctx;

typedef enum {
  HW_OK = 0,
  HW_EINVAL = 1,     /* invalid argument (checked on the host before any launch)        */
  HW_ENOMEM = 2,     /* device or host allocation failed during setup                   */
  HW_ECUDA = 3,      /* a CUDA runtime / cuBLAS call failed                              */
  HW_ESTATE = 4,     /* call out of order (no basis, no potential, no device, ...)       */
  HW_ENOTCONV = 5,   /* eigensolver reached maxit; partial results are returned          */
  HW_ETIMEOUT = 6    /* a bounded device-side wait gave up; the context stays usable     */
} hw_status;

typedef enum {
  HW_FP64 = 0,       /* every step in FP64                                                 */
  HW_MIXED = 1,      /* transforms in FP32 (FP32 accumulate); diagonal terms, Gram,
                        Cholesky, Rayleigh-Ritz and the final residual check in FP64      */
  HW_FP64_DF = 2     /* hw_apply_H only: FP64 blocks and diagonal term; the radial and
                        angular transforms (Algorithms 1-4 with the potential multiply) in
                        double-float arithmetic -- pairs of FP32 numbers, about 48
                        significant bits, on the FP32 pipe -- on the 64 x 48 grid with at most
                        16 consecutive kept m rows and nu = 0 (other cases: as HW_FP64).  What
                        the mixed-precision solver uses for its FP64 H X (HW_OPT_FP64_HX).  */
} hw_prec;

typedef enum {
  HW_PRECOND_TPA = 0,      /* Teter-Payne-Allan diagonal (Sec. Eigensolvers and Preconditioning) */
  HW_PRECOND_LEARNED = 1,  /* per-mode MLP scaling installed by hw_set_mlp                       */
  HW_PRECOND_NONE = 2
} hw_precond_kind;

/* Geometry and discretisation (Secs. "Description of Physical System", "Wave function
 * storage", "Imposition of kinetic energy cutoff").  The basis box follows the grids:
 * M = floor((N_th1-1)/s), N = floor((N_th2-1)/s), K = floor(N_r/s) with s = oversample
 * (the paper's grid rule N_th = 4*max+1, N_r = 4*K_max read backwards). */
typedef struct {
  double R;          /* cylinder radius (Dirichlet wall), bohr, > 0                        */
  double tau;        /* screw pitch, bohr, > 0                                              */
  double alpha;      /* twist per pitch (turns)                                             */
  int ncyc;          /* cyclic order Ncyc >= 1                                              */
  double ecut;       /* kinetic cutoff, Hartree; <= 0 keeps the whole box                   */
  int Nr;            /* radial Gauss-Jacobi nodes, >= oversample                            */
  int Nth1;          /* theta1 Fourier nodes; factors 2 and 3 only; >= 2M+1                 */
  int Nth2;          /* theta2 Fourier nodes; factors 2 and 3 only; >= 2N+1                 */
  int oversample;    /* s >= 2                                                              */
} hw_basis_params;

/* Create a context on CUDA device `device` whose calls are ordered on `cuda_stream` (a
 * cudaStream_t, NULL = legacy default stream).  device = -1 creates a host-only context:
 * hw_setup_basis and the hw_get_* queries work, every device call returns HW_ESTATE. */
hw_status hw_create(hw_ctx** out, int device, void* cuda_stream);
void hw_destroy(hw_ctx* ctx);
const char* hw_last_error(const hw_ctx* ctx);

/* Basis set, radial quadrature, tables and cutoff masks for nk points (eta_b, nu_b)
 * (eqs. Phi_expanded_in_basis_set, Basis_fun_derived, Energy_cutoff; Sec. eta-space
 * discretization).  ecut_per_k (host, nullable) overrides params->ecut per point.
 * nu (host, [nk], nullable = all 0): the cyclic wavenumbers, physically 0 .. Ncyc-1 (any
 * finite value is accepted).  For nu != 0 H carries the 1/r^2 terms of eqs. ell_mnk and
 * I_nkk_prime; their radial integrals are tabulated here per |n| (a Gauss-Jacobi rule fine
 * enough for the Bessel products).  For n = 0 that integral diverges at r = 0 (J_0 does not
 * vanish there), and the table takes the value of the transform's radial rule instead: the
 * n = 0 modes of a nu != 0 point are then a finite but grid-dependent approximation.
 * L_out (host, [nk]) receives the masked basis sizes.  Replaces any earlier basis. */
hw_status hw_setup_basis(hw_ctx* ctx, const hw_basis_params* params, int nk, const double* eta,
                         const double* nu, const double* ecut_per_k, int64_t* L_out);

/* Sizes: box limits, grid point count N_th1*N_th2*N_r, number of (m, n) angular pairs kept
 * at any of the k-points. Any pointer may be NULL. */
hw_status hw_get_sizes(const hw_ctx* ctx, int* M, int* N, int* K, int64_t* grid_points,
                       int* n_pairs);

/* Radial nodes r_p (ascending) and weights omega_p with sum_p omega_p f(r_p) ~ int_0^R f r dr
 * (host outputs, [Nr] each; either may be NULL). */
hw_status hw_get_grid(const hw_ctx* ctx, double* r_nodes, double* r_weights);

/* (m, n, k) of every kept mode of k-point k in compact order, k 0-based (host, [3*L_k]). */
hw_status hw_get_index_map(const hw_ctx* ctx, int k, int32_t* mnk);

/* Diagonal of the Hamiltonian's reciprocal-space part at k-point k, i.e. the shifted kinetic
 * energy 1/2 lambda^0 - a - b(i2pi m) - c(i2pi n Ncyc) of Algorithm 5 (host, [L_k]). */
hw_status hw_get_kinetic(const hw_ctx* ctx, int k, double* ke);

/* Radial table xi_{n,k}(r_p) for angular order n (host output [Nr*K], p-major). */
hw_status hw_get_radial_table(const hw_ctx* ctx, int n, double* table);

/* Table I(n, k, k') of eq. I_nkk_prime for angular order n (host output [K*K], symmetric),
 * the radial integral of the nu != 0 terms: (nu^2 - 2 nu n Ncyc)/R^2 I(n, k, k') couples the
 * coefficients (m, n, k) and (m, n, k').  For n = 0 the integral diverges; the value returned
 * (and used) is that of the transform's radial rule (see hw_setup_basis). */
hw_status hw_get_itable(const hw_ctx* ctx, int n, double* table);

/* Install the real potential V on the grid (eq. wavefun_storage_real order, length
 * N_th1*N_th2*N_r).  on_device != 0: V is a device pointer (copied on the stream), else a
 * host pointer (copied synchronously). */
hw_status hw_set_potential(hw_ctx* ctx, const double* V, int on_device);

/* Build and install the Gaussian-well potential
 *   V(x) = sum_a sum_{zeta,mu} -Z_a exp(-|x - Upsilon_{zeta,mu} x_a|^2 / (2 sigma_a^2))
 * summed over the images of the helical group (eq. symm_opera) with |z - z_image| <= 10 sigma.
 * atoms: host array [n_atoms][5] of (r, vartheta, z, Z, sigma).  Evaluated once per potential
 * in FP64 on the host's cores (std::thread), then installed as by hw_set_potential; returns when
 * V is installed (host-only contexts only evaluate it).  V_out (host, nullable) receives V in
 * eq. wavefun_storage_real order. */
hw_status hw_build_potential(hw_ctx* ctx, int n_atoms, const double* atoms, double* V_out);

/* Y = H X at k-point k (Algorithm 5): reciprocal-space diagonal terms, inverse transform
 * (Algorithms 1-2), pointwise V, forward transform (Algorithms 3-4), and for nu != 0 the
 * 1/r^2 terms (nu^2 - 2 nu n Ncyc)/R^2 I(n, k, k') within each (m, n) (the I_n loop).  X, Y: device,
 * complex128, L_k x ns, leading dimension ld.  X and Y must not overlap. */
hw_status hw_apply_H(hw_ctx* ctx, int k, const double* X, double* Y, int ns, int64_t ld,
                     hw_prec prec);

/* The same product as hw_apply_H for callers that cannot allocate device memory (a budget
 * fixed at start-up, or places where cudaMalloc is not allowed or would synchronise).  No
 * counterpart in the paper.  The call allocates nothing: its intermediates live in one
 * file-scope device array of 64 MiB that every GPU loading this library holds until exit,
 * resolved with cudaGetSymbolAddress on the first call on each device (make that first call
 * before any stream capture).  Columns are processed in passes that fit the array; a basis
 * whose single column does not fit (2 * N_r * n_pairs complex values) is rejected with
 * HW_EINVAL.  Calls share the array: calls that overlap on the GPU race and must be ordered
 * by the caller.  The array's address is resolved once per device for the life of the
 * process, so resetting a device (cudaDeviceReset) while this library is loaded is not
 * supported.  Arguments as for hw_apply_H; X and Y must not overlap at all (HW_EINVAL). */
hw_status hw_apply_H_noalloc(hw_ctx* ctx, int k, const double* X, double* Y, int ns, int64_t ld,
                             hw_prec prec);

/* Y_b = H(b) X_b for the nk k-points kidx[0..nk) in one pipeline; X[b], Y[b] are device
 * pointers to L_{kidx[b]} x ns blocks with leading dimension ld (>= max L). */
hw_status hw_apply_H_batched(hw_ctx* ctx, int nk, const int* kidx, const double* const* X,
                             double* const* Y, int ns, int64_t ld, hw_prec prec);

/* Z = K R, a diagonal preconditioner at k-point k applied column by column (device,
 * complex128, L_k x ns, leading dimension ld; Z may equal R).  kind = HW_PRECOND_TPA: the
 * Teter-Payne-Allan diagonal P(g)/(P(g)+16 g^4), P = 27+18g+12g^2+8g^3, g_i = KE_i / KE_res,
 * KE_res the |r_i|^2-weighted mean of KE_i over the column (Sec. Eigensolvers and
 * Preconditioning).  kind = HW_PRECOND_LEARNED: Z_i = s(features_i, ritz_j) R_i with the MLP
 * of hw_set_mlp; ritz is a device array [ns] (required for LEARNED, ignored otherwise). */
hw_status hw_apply_precond(hw_ctx* ctx, int k, const double* R, double* Z, int ns, int64_t ld,
                           const double* ritz, int kind);

/* Lowest n_eig eigenpairs at the nk k-points kidx[] by block LOBPCG (Sec. Eigensolvers and
 * Preconditioning), or by Chebyshev-filtered subspace iteration (HW_OPT_EIGENSOLVER), on blocks
 * of `block` >= n_eig columns (0: n_eig + max(4, n_eig/8) for LOBPCG, n_eig + max(8, 3 n_eig/16)
 * for the Chebyshev solver),
 * at most 112 columns (HW_EINVAL above: the Cholesky-QR keeps its factor in shared memory).
 * More than HW_OPT_WINDOW eigenpairs (default 80) are solved in w = ceil(n_eig / window)
 * consecutive windows of ceil(n_eig / w) eigenpairs (the last one the rest).  Each window is a
 * block solve as above (`block` then applies to one window; default the window plus
 * max(32, window / 2) buffer columns, at most 112 and L_min / 3) restricted to the orthogonal
 * complement of the eigenvectors the earlier windows converged: the start block and, every
 * iteration, the new search directions (LOBPCG) or the filtered block (Chebyshev) are
 * projected against them (in FP64; in the FP32 and hybrid phases of the mixed form with FP32
 * products).  Windows before the last aim at tol / 2 (their residuals leak into the later
 * windows' eigenvectors, which the projection cannot remove) and are accepted at tol once
 * their residuals stop falling.  The windows run in lockstep over the k-points; X0 must be
 * NULL then (HW_EINVAL); iters is the sum over the windows.
 * A column is converged when ||H x - theta x||_2 <= tol with ||x|| = 1.  X0 (nullable):
 * nk device pointers to L_k x block complex128 start blocks (leading dimension L_k); NULL
 * draws a seeded Gaussian start on the device.  Outputs: evals (host, [nk*n_eig]), iters
 * (host, [nk], nullable), resid (host, [nk*n_eig], nullable: final residual norms),
 * evecs (nullable: nk device pointers to L_k x n_eig blocks with leading dimension ld_evecs).
 * Returns HW_ENOTCONV (with the partial results) when maxit is reached.  Synchronous. */
hw_status hw_solve_eigs(hw_ctx* ctx, int nk, const int* kidx, int n_eig, int block, double tol,
                        int maxit, hw_prec prec, int precond_kind, const double* const* X0,
                        double* evals, double* const* evecs, int64_t ld_evecs, int* iters,
                        double* resid);

/* ---- learned per-mode preconditioner (an extension refining the TPA diagonal) ----------
 * Network: x_i = [KE_i/10, (m-eta)/M, (n Ncyc-nu)/N, k/K, theta/10, Vd_i/10] (Hartree),
 * o_i = w3 . silu(W2 silu(W1 x_i + b1) + b2) + b3, scaling s_i = tpa_i exp(o_i) with tpa_i the
 * TPA factor of the column; Vd_i is the potential's diagonal in mode i (angular mean of V on
 * each radial node integrated against xi_{n,k}^2).  Parameters: 4673 FP32 values laid out as
 * W1[64][6] | b1[64] | W2[64][64] | b2[64] | w3[64] | b3; inference and training use their
 * BF16 roundings with FP32 accumulation; the FP32 values are the Adam master copy. */

/* Install (host FP32 array of n = 4673 values) and reset the optimiser state. */
hw_status hw_set_mlp(hw_ctx* ctx, const float* params, int64_t n);

/* Copy the current FP32 parameters to the host (n = 4673). */
hw_status hw_get_mlp(hw_ctx* ctx, float* params, int64_t n);

/* Vd_i of every kept mode of k-point k (host [L_k]); needs a network and a potential. */
hw_status hw_get_potential_diagonal(hw_ctx* ctx, int k, double* vd);

/* Training loss of a batch of ns columns at k-point k: mean over columns of
 * 1 - |<s.R, E>|^2 / (|s.R|^2 |E|^2).  R (residuals) and E (target corrections): device
 * complex128 L_k x ns blocks, leading dimension ld; ritz: host [ns] Ritz values; vdiag: device
 * [L_k] potential diagonal of the batch's potential (NULL: the installed potential's).
 * loss: host scalar; grad (nullable): host [4673] gradient w.r.t. the parameters. */
hw_status hw_mlp_loss_grad(hw_ctx* ctx, int k, const double* R, const double* E,
                           const double* ritz, int ns, int64_t ld, const double* vdiag,
                           double* loss, float* grad);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, step size lr) on the same batch loss;
 * loss (host, nullable) receives the loss before the step. */
hw_status hw_mlp_train_step(hw_ctx* ctx, int k, const double* R, const double* E,
                            const double* ritz, int ns, int64_t ld, const double* vdiag,
                            float lr, double* loss);

/* hw_solve_eigs at one k-point that also records training data: at the iterations rec_iters
 * [n_rec] it stores the residual block R (device rec_R, [n_rec][block][ld] complex128), the
 * Ritz values and residual norms (host rec_theta / rec_res, [n_rec][block]); after
 * convergence it stores in rec_E the target correction of every recorded column,
 * e_j = (I - X X^H) X* X*^H x_j, with X the recorded block and X* the converged n_eig
 * eigenvectors.  Entries of iterations never reached are left untouched. */
hw_status hw_solve_eigs_traced(hw_ctx* ctx, int k, int n_eig, int block, double tol, int maxit,
                               hw_prec prec, int precond_kind, const double* X0, int n_rec,
                               const int* rec_iters, double* rec_R, double* rec_E,
                               double* rec_theta, double* rec_res, int64_t ld, double* evals,
                               int* iters);

/* Residual history of the last hw_solve_eigs (metrics; the paper plots such histories for its
 * LOBPCG + TPA runs, Sec. "Eigensolvers and Preconditioning"): for k-point k, one entry per
 * filter cycle or LOBPCG iteration (windows follow each other), phase[i] its HW_HIST_* code and
 * res[i] the largest residual ||H x - theta x|| over the wanted columns at its start.  Writes
 * min(n, max_n) entries (phase and res may be NULL) and the count n to *n_out (0 when k took no
 * part).  Host arrays; no device work. */
enum {
  HW_HIST_FILTER_FP32 = 0,    /* Chebyshev filter cycle, FP32 H X and products */
  HW_HIST_FILTER_FP64 = 1,    /* Chebyshev filter cycle, FP64 */
  HW_HIST_LOBPCG_FP32 = 2,    /* LOBPCG iteration, FP32-class products */
  HW_HIST_LOBPCG_HYBRID = 3,  /* LOBPCG iteration, FP64-class products for X only */
  HW_HIST_LOBPCG_FP64 = 4     /* LOBPCG iteration, FP64-class products */
};
hw_status hw_get_residual_history(hw_ctx* ctx, int k, int* phase, double* res, int max_n, int* n_out);

/* Self-test of the bounded device wait (no counterpart in the paper; failure detection).  The
 * library's grid-wide barrier (used by the FP64 Jacobi eigensolver) gives up after a bounded
 * number of polls, sets the device status word to HW_ETIMEOUT and lets every CTA leave, so a
 * barrier that can never complete ends the kernel instead of hanging the GPU.  This call runs
 * three such barriers over `nblocks` co-resident CTAs (2 .. SM count) with a wait bound of
 * `spin_limit` polls of 100 ns (1 .. 2^24); CTA `skip_block` (-1: none) leaves before the first
 * barrier, so the others can never be released.  On return *wait_status (host) holds the
 * kernel's status word: HW_OK when every barrier completed, HW_ETIMEOUT when a wait ran out.
 * Synchronises the context's stream.  Returns HW_EINVAL for arguments out of range. */
hw_status hw_selftest_barrier(hw_ctx* ctx, int nblocks, long long spin_limit, int skip_block,
                              int* wait_status);

/* The eigensolver's Cholesky factorisation on its own (the factor step of its Cholesky-QR
 * orthonormalisation, Sec. "Eigensolvers and Preconditioning"): G = L L^H for nprob Hermitian
 * positive definite n x n matrices.  G: device, complex128 column-major, problem b at
 * G + 2 n^2 b doubles, only its lower triangle read, overwritten (used as scratch); L: device,
 * same layout, distinct from G, receives the lower factor with zeros above the diagonal.
 * prec: HW_FP64 (FP64 arithmetic) or HW_MIXED (FP32 arithmetic, as in the mixed solver's first
 * phase; n <= 160).  n <= 112 runs the unblocked kernel (one barrier per column), larger n
 * the blocked one.  fail: host [nprob]: 0, or 1 + the column of the first pivot that is not
 * positive and finite (that problem's L is then not a factor).  1 <= nprob <= 64.
 * Synchronous. */
hw_status hw_cholesky(hw_ctx* ctx, int n, int nprob, double* G, double* L, int* fail, hw_prec prec);

/* The Rayleigh-Ritz step's dense Hermitian eigensolver on its own (Sec. "Eigensolvers and
 * Preconditioning": the small projected eigenproblem of LOBPCG).  A: device, nprob Hermitian
 * n x n complex128 matrices (column-major, contiguous, n even, read only); w: device
 * [nprob][n] eigenvalues ascending; Z: device [nprob][n][n] eigenvector columns.  method 0:
 * FP64 parallel Jacobi (all n pairs).  method 1: FP32 Householder tridiagonalisation,
 * bisection and inverse iteration, then FP64 refinement of the lowest nw pairs (only the first
 * nw entries of w and columns of Z are FP64-accurate; n <= 236).  Synchronous. */
hw_status hw_heev(hw_ctx* ctx, int n, int nprob, int nw, const double* A, double* w, double* Z,
                  int method);

/* Electron density on the real-space grid (Sec. "Convergence Studies", the electron-density
 * equation): rho = (2 / Ncyc) sum_b w[b] sum_j occ[b*ns + j] |phi_{b,j}|^2, where phi_{b,j} is the
 * inverse basis transform (eq. Naive_Inverse_Transform, by Algorithms 1-2) of column j of the
 * state block X[b] at k-point kidx[b] (the sum over (eta, nu) points is the sum over b, with the
 * weights w; for Ncyc > 1 pass every nu).  X: nk device
 * pointers to complex128 L_k x ns blocks with leading dimension ld; occ: host [nk*ns]
 * occupations; w: host [nk] k-point weights (the Monkhorst-Pack weights 1/N_eta for a uniform
 * set); rho: device, N_th1*N_th2*N_r doubles in eq. wavefun_storage_real order (the order of
 * hw_set_potential), overwritten.  prec: HW_FP64 transforms, or HW_MIXED (FP32 transforms and
 * FP32 accumulation of |phi|^2, FP64 sum over CTAs).  HW_EINVAL when one radial node's
 * accumulator and transform buffers exceed 200 KB of shared memory at that precision (the
 * 192 x 96 nanowire grid in FP64; its mixed density fits).  Synchronous.  The column weights
 * are kept in a small device array of the context (allocated on first use, grown when
 * needed). */
hw_status hw_density(hw_ctx* ctx, int nk, const int* kidx, const double* const* X, int ns, int64_t ld,
                     const double* occ, const double* w, double* rho, hw_prec prec);

/* Cartesian gradient on the real-space grid of E = sum Ehat_{m,n,k} F_{m,n,k} (Appendix C) for
 * each of the ns coefficient columns X (device, complex128, L_k x ns, leading dimension ld,
 * compact order of k-point k; no Bloch phase is applied): E_theta1 and E_theta2 are inverse
 * transforms of (i 2 pi m) Ehat and (i 2 pi n Ncyc) Ehat (eq. Derivative_of_energy_wrt_theta),
 * E_r the inverse transform with the radial derivative of the basis (eqs. E_r, B_r), combined by
 * the chain rule of eq. Cartesian_Derivatives.  D: device, complex128, ns x 3 x N_th1 x N_th2 x
 * N_r: for column c the components x, y, z, each in eq. wavefun_storage_real order (the order of
 * hw_set_potential).  prec: HW_FP64 transforms, or HW_MIXED (FP32 radial and angular
 * transforms, FP64 chain rule and output).  Asynchronous on the context's stream.  HW_EINVAL
 * when one radial node's transform buffers exceed 200 KB of shared memory at that precision. */
hw_status hw_gradient(hw_ctx* ctx, int k, const double* X, int ns, int64_t ld, double* D, hw_prec prec);

/* Gram product of the eigensolver's mixed form (Sec. "Eigensolvers and Preconditioning": the
 * Rayleigh-Ritz matrices S^H H S and the orthogonalisations): C_b = A_b^H B_b for nprob
 * problems, A_b: K x m, B_b: K x n complex128 column-major device blocks (leading dimensions
 * lda, ldb >= K; problem b at A + b*sA, B + b*sB elements), C_b: m x n (ldc >= m, stride sC).
 * Products in FP32 (inputs rounded to nearest), accumulation in FP64 every 32 rows; chunk
 * partials reduced in a fixed order (deterministic).  Asynchronous on the context's stream.
 * HW_EINVAL on bad sizes (m, n <= 512, 1 <= nprob <= 64). */
hw_status hw_gram(hw_ctx* ctx, int m, int n, int K, int nprob, const double* A, int64_t lda, int64_t sA,
                  const double* B, int64_t ldb, int64_t sB, double* C, int64_t ldc, int64_t sC);

/* Block product of the eigensolver (Sec. "Eigensolvers and Preconditioning": Gram matrices,
 * Rayleigh-Ritz projections, block updates) on the tensor cores: for b < batch,
 *   C_b = alpha op(A_b) B_b + beta C_b,   op(A) = A^H (transA = 1, A_b: k x m) or A (0, m x k),
 * B_b: k x n, C_b: m x n; complex128, column-major device blocks with leading dimensions lda,
 * ldb, ldc and batch strides sA, sB, sC (complex elements).  Every real row of op(A) and of B
 * (complex entries as interleaved real pairs) is scaled by a power of two and cut into BF16
 * integer digits; the digit products are summed by tcgen05 MMAs in TMEM.  cls 0 (FP64 class):
 * 8 digits of 7 bits, exact group sums added into a 64-bit fixed point, error below
 * 2^-46 max|op(A)_i,:| max|B_:,j| per reduction element (tighter than an FP64 GEMM's bound for
 * vectors without a wide dynamic range); cls 1 (FP32 class): every operand as a TF32 pair
 * hi + lo, the products hi hi' + hi lo' + lo hi' summed in FP32 by tcgen05 kind::tf32 MMAs,
 * about 2^-22 of the same scale.  Deterministic (fixed-order split reduction).  The library
 * grows a workspace for the planes (up to 1 GiB; larger batches run in chunks).
 * cls 2 and 3: the small-product kernel instead (every extent below 1024, no workspace): SIMT
 * on the FP32 pipe, one CTA per 8 x 8 output tile with a four-way split of each reduction
 * added in a fixed order; cls 2 rounds the FP64 operands to double-float pairs (~48-bit
 * significands, error ~2^-44 of sum |op(A)||B|), cls 3 to FP32.
 * Asynchronous on the context's stream.  HW_EINVAL on bad sizes (n <= 4096, m, k <= 2^20;
 * below 1024 for cls 2, 3). */
hw_status hw_block_product(hw_ctx* ctx, int transA, int m, int n, int k, double alpha, const double* A,
                           int64_t lda, int64_t sA, const double* B, int64_t ldb, int64_t sB, double beta,
                           double* C, int64_t ldc, int64_t sC, int batch, int cls);

/* Autotune the H X kernels' tile shapes for blocks of ns columns at k-point k: the slab
 * kernel's theta2 chunk and the number of columns per pass are timed (CUDA events, best of
 * 2 after a warm-up) for every candidate in FP64 and FP32 and the fastest are kept for later
 * calls.  results (host, nullable): up to max_results rows of 4 floats (precision 0/1, chunk,
 * pass columns, milliseconds); n_results receives the row count.  Allocates two temporary
 * blocks; synchronous. */
hw_status hw_autotune(hw_ctx* ctx, int k, int ns, float* results, int max_results,
                      int* n_results);

/* Options of a context. */
typedef enum {
  HW_OPT_RR_METHOD = 0,     /* Rayleigh-Ritz eigensolver: 0 auto (Householder FP32 + FP64
                               refinement when n <= 236, checked, with the FP64 Jacobi as the
                               retry), 1 FP64 Jacobi always.  Default 0. */
  HW_OPT_RR_FALLBACKS = 1,  /* read only: Householder results rejected by the check so far */
  HW_OPT_LOWP_SWITCH = 2,   /* mixed form only: the block products over the basis dimension
                               (Gram matrices, projections, block updates) run in complex FP32
                               until every wanted residual is below 10^-value (or the residuals
                               stop falling: FP32 products stall near 1e-5), then in FP64 (X
                               re-orthonormalised, H X recomputed in FP64, P restarted).
                               0 disables (FP64 throughout); 1..12; default 5. */
  HW_OPT_GRAM_KERNEL = 3,   /* mixed form, FP32-product phase only: 1 forms the products
                               A^H B over the basis dimension with hw_gram's kernel (FP32
                               products, FP64 accumulation every 32 rows); 0 (default) leaves
                               them to HW_OPT_TC_GEMM's route (the tensor-core kernel), measured
                               faster on the tube. */
  HW_OPT_HYBRID = 4,        /* mixed form, FP64 phase: 1 (default) first keeps FP64 only for
                               the products that involve X (its rows of the Rayleigh-Ritz matrix,
                               its share of the X / H X updates, one projection of W and of P
                               against X) and forms the rest of the W and P orthogonalisation,
                               their Gram block and the P update in FP32; such residuals stall
                               near 3e-7, so when the best residual has not dropped by 30% in 4
                               iterations every product becomes FP64.  0: FP64 throughout the
                               phase. */
  HW_OPT_EIGENSOLVER = 5,   /* block eigensolver of hw_solve_eigs: 0 (default) LOBPCG with the
                               preconditioner; 1 Chebyshev-filtered subspace iteration: filter +
                               Rayleigh-Ritz cycles (HW_FP64: to the end; HW_MIXED: with FP32
                               products until the FP32 phase ends, then LOBPCG's mixed form with
                               the preconditioner finishes from the filtered block).  iters and
                               maxit count cycles plus LOBPCG iterations. */
  HW_OPT_CHEB_DEGREE = 6,   /* Chebyshev filter degree (H X products per cycle), 2..64;
                               default 24; the maximum when HW_OPT_CHEB_ADAPT is on. */
  HW_OPT_CHEB_ADAPT = 7,    /* 1 (default): each FP64 cycle takes the smallest degree (at most
                               HW_OPT_CHEB_DEGREE) estimated to bring every unconverged wanted
                               residual to tol; 0: always the full degree. */
  HW_OPT_CHEB_LOCK = 8,     /* 1 (default): leading Ritz columns whose residuals are below half
                               the phase's target are not filtered (soft locking); 0: every
                               column is filtered every cycle. */
  HW_OPT_SLAB_KERNEL = 9,   /* angular kernel on the 64 x 48 grid (Algorithms 2 and 4 with the
                               potential multiply): 2 (default) every transform in registers for
                               FP32 -- theta2 as 4 lanes x 12-point DFTs joined by a 4-point DFT
                               across the lanes, theta1 as 4 lanes x 16-point DFTs, several
                               slabs per CTA -- and for FP64 the 1 kernel; 3 the register kernel
                               in both precisions; 1 the theta1 transforms split 64 = 4 x 16 over
                               the 4 lanes of a theta2 point with Stockham theta2 passes in
                               shared memory; 0 the Stockham FFTs throughout.  The register
                               kernel needs at most 16 kept m rows, consecutive in m; other
                               bases take 1.  Every other grid uses the Stockham FFTs. */
  HW_OPT_TAIL_NO_P = 10,    /* Chebyshev solver, mixed form: 1 starts the LOBPCG end phase
                               without conjugate directions (Rayleigh-Ritz on [X W], each
                               iteration cheaper) and switches them on for good once an
                               iteration fails to halve the largest wanted residual; 0 (default):
                               with them from the start (over 8 start blocks of the tube
                               workload: 8-10 end-to-end iterations against 9-14). */
  HW_OPT_WINDOW = 11,       /* hw_solve_eigs: largest number of eigenpairs one block solves,
                               1..100; 0 (default) means 80.  More eigenpairs than this are
                               solved in consecutive windows of equal size (see hw_solve_eigs). */
  HW_OPT_TC_GEMM = 12,      /* the eigensolver's block products: 1 (default) the tensor-core
                               kernel of hw_block_product (FP64 class in the FP64 phases, FP32
                               class in the FP32-product phase) for every product with an extent
                               over the basis dimension (m or k >= 1024), the small dense
                               products of the Rayleigh-Ritz step as HW_OPT_SMALL_GEMM says; 2 the
                               tensor-core kernel for every product; 0 cuBLAS over the basis
                               dimension (ZGEMM, or CGEMM on FP32 copies). */
  HW_OPT_RADIAL_KERNEL = 13, /* radial transforms of the mixed-precision H X: 1 (default) on
                               the tensor cores (both operands split into three BF16 parts, the
                               six part products as tcgen05 MMAs, the leading one in its own TMEM
                               accumulator; one CTA per 64 (column, pair) items of an |n| group;
                               the forward kernel of launches with nu != 0 stays on the FP32 SIMT
                               kernel); 0 the FP32 SIMT kernels.  FP64 H X always uses the FP64
                               SIMT kernels. */
  HW_OPT_FP64_HX = 14,      /* the FP64 H X of a HW_MIXED solve (its hand-over to FP64 products
                               and the FP64 check of every convergence claim): 1 (default) the
                               angular transforms in double-float arithmetic (as hw_apply_H with
                               HW_FP64_DF), 0 in FP64.  HW_FP64 solves always use FP64. */
  HW_OPT_SMALL_GEMM = 15,   /* the eigensolver's small products (every extent below 1024: the
                               Rayleigh-Ritz refinement, the Newton-Schulz steps): 1 (default)
                               the library's SIMT kernel for the FP32 class (FP64 operands
                               rounded to FP32, as hw_block_product class 3) and, inside
                               HW_MIXED solves, for the FP64 class in double-float (class 2: its
                               ~1e-14 errors, divided by eigenvalue gaps in the first-order
                               refinement, leave the refined Ritz vectors orthonormal to ~1e-11,
                               within the solver's 1e-9 check); HW_FP64 solves and hw_heev take
                               cuBLAS ZGEMM for the FP64 class; 2 the SIMT kernel for both classes
                               everywhere; 0 cuBLAS for both. */
  HW_OPT_OVERLAP_LAUNCH = 16 /* the FP32 H X's three kernels (tensor-core radial inverse, register
                               slab, tensor-core radial forward): 1 (default) launched with
                               programmatic stream serialisation, so that each starts its CTAs
                               while the one before it drains and waits on the device for that
                               kernel's results (the same order and results as 0); 0 plain
                               stream-ordered launches.  The library's other kernels always use
                               such launches, each waiting for the kernel before it before it
                               reads or writes anything (again the order and results of plain
                               launches), except the cooperative Jacobi kernels and the gradient
                               kernel. */
} hw_option;
/* Set an option (HW_EINVAL for an unknown option, a read-only one or a bad value). */
hw_status hw_set_option(hw_ctx* ctx, int option, int value);
/* Read an option or counter into *value. */
hw_status hw_get_option(hw_ctx* ctx, int option, long long* value);

/* Wait for all work on the context's stream. */
hw_status hw_synchronize(hw_ctx* ctx);

/* Phases timed by the profiler (CUDA events recorded on the context's stream around each
 * launch of the phase; device time, not host time). */
typedef enum {
  HW_PH_RADIAL_INV = 0,   /* gather + inverse radial transform (Algorithm 1, first loop)   */
  HW_PH_SLAB = 1,         /* angular FFTs with the potential multiply (Algorithms 2, 4)     */
  HW_PH_RADIAL_FWD = 2,   /* forward radial quadrature + diagonal + scatter (Algorithm 3)   */
  HW_PH_PRECOND = 3,      /* diagonal preconditioner                                        */
  HW_PH_GEMM = 4,         /* block products of the eigensolver (tensor-core, small-product
                             and, where an option selects it, cuBLAS kernels)               */
  HW_PH_CHOL = 5,         /* Cholesky factorisations + triangular solves                    */
  HW_PH_EIG = 6,          /* rest of the Rayleigh-Ritz eigensolver (eigenvalues, vectors,
                             FP64 refinement)                                               */
  HW_PH_OTHER = 7,        /* residuals, gathers, padding                                     */
  HW_PH_MLP = 8,          /* preconditioner network (inference and training)                 */
  HW_PH_TRIDIAG = 9,      /* Householder reduction of the Rayleigh-Ritz matrix (FP32)        */
  HW_PH_DENSITY = 10,     /* inverse angular passes and |phi|^2 accumulation of hw_density  */
  HW_PH_GRADIENT = 11,    /* inverse angular passes and chain rule of hw_gradient          */
  HW_NPHASE = 12
} hw_phase;

/* Turn per-phase profiling on (enable != 0) or off; either resets the accumulators.  While on,
 * every phase launch is bracketed by CUDA events (small overhead). */
hw_status hw_profile(hw_ctx* ctx, int enable);

/* Synchronize the stream and read the accumulated device milliseconds and launch counts per
 * phase (host arrays of HW_NPHASE entries; either may be NULL). */
hw_status hw_profile_read(hw_ctx* ctx, double* ms, int64_t* count);

/* Algorithmic work accumulated per phase since profiling was turned on (host array of
 * HW_NPHASE entries): real floating-point operations of the method for HW_PH_TRIDIAG
 * ((16/3) n^3 per n x n problem) and HW_PH_CHOL ((8/3) n^3 per factorisation plus 4 rows n^2
 * per triangular solve of rows x n); zero for the other phases. */
hw_status hw_profile_work(hw_ctx* ctx, double* work);

/* Number of this library's own kernels launched on the context's stream since creation
 * (cuBLAS kernels are not counted). */
int64_t hw_launch_count(const hw_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* HELICWAVE_H */

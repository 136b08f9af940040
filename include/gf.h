/*
 * gf.h -- C-ABI of libgf, the GB300 (sm_103a) lattice Green's function library.
 *
 * The library evaluates the data-parallel hot path of the fully charge
 * self-consistent LDA+DMFT loop of Zhao et al., "Implementation of LDA+DMFT
 * with pseudo-potential-plane-wave method" (arXiv:1111.2157):
 *
 *   G(k, i w_n)  = [(i w_n + mu) I - H_k - P_k^+ Sigma(i w_n) P_k]^{-1}   Sec. 3.2.2, Eq. dmftloop1
 *   G_loc(i w_n) = sum_k w_k P_k G(k, i w_n) P_k^+                      Sec. 3.2.2, k-sum in Eq. dmftloop2
 *   rho_k        = (1/beta) sum_n G(k, i w_n) e^{i w_n 0+}               Sec. 3.3, Eq. rho_LDA+DMFT
 *   N(mu)        = sum_k w_k Tr rho_k = N_target                        Sec. 3.3, Eq. fix_mu
 *   n_corr       = sum_k w_k Tr(P_k rho_k P_k^+)                        Sec. 3.4, Eq. nf_LDA+DMFT
 *
 * Conventions shared by every entry point:
 *  - w_n = (2n+1) pi / beta, n = 0 .. n_iw-1 (positive fermionic frequencies only;
 *    the negative ones follow from G(-i w_n) = G(i w_n)^+, which needs
 *    Sigma(-i w_n) = Sigma(i w_n)^+).
 *  - The Matsubara sum subtracts the 1/(i w) and 1/(i w)^2 moments of G,
 *    T = I/(i w) + M2/(i w)^2 with M2 = H_k + P_k^+ Sigma_inf P_k - mu I, and adds
 *    their exact sums back: rho_k = (1/beta) sum_{n<n_iw} [(G-T) + (G-T)^+] + I/2
 *    - (beta/4) M2.  tail_order = 1 keeps only the 1/(i w) moment.
 *  - The band index n already includes spin (Sec. 3.1): no factor 2 anywhere.
 *  - Complex numbers are interleaved (re, im).  Arrays are row-major.
 *  - Energies in eV, beta in 1/eV.
 *  - k-points are grouped by system: k_system[] must be non-decreasing.
 *  - Inputs of several systems are packed system after system.  With
 *    gf_desc.system_dtype each system's block is stored in that system's dtype
 *    (complex128: 16 bytes, complex64: 8 bytes per number), so one context
 *    holds complex128 and complex64 systems; complex64 numbers are widened
 *    exactly on the device.
 *  - Pointer arguments named *_ptr may point to host memory (pageable or
 *    pinned) or to device memory of the context's device; the library tells
 *    them apart through unified addressing.  Input arrays are copied into
 *    library-owned device memory; the caller keeps ownership of its buffers.
 *  - Every compute call is ordered on the context's stream and returns after
 *    the stream has drained, so host outputs are valid on return.
 *  - Calls on one context are not thread-safe.  No entry point throws; each
 *    returns a gf_status and records a message for gf_last_error().  A host
 *    allocation that fails inside the library returns GF_ENOMEM (gf_create
 *    then frees what it had built and leaves *out NULL).
 *  - There is no CPU fallback: gf_create fails with GF_ECUDA without a device.
 */
#ifndef GF_H
#define GF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gf_ctx gf_ctx;

typedef enum {
    GF_OK = 0,
    GF_EINVAL = 1,     /* invalid argument (sizes, pointers, enum values)          */
    GF_ENOMEM = 2,     /* device or host allocation failed                         */
    GF_ECUDA = 3,      /* a CUDA runtime call failed (message in gf_last_error)    */
    GF_ESINGULAR = 4,  /* a zero or non-finite pivot in some (k, i w_n) inverse    */
    GF_ENOTCONV = 5,   /* a mu search missed tol in max_iter, or Jacobi its sweep cap */
    GF_ETIMEOUT = 6,   /* a bounded wait of the tensor-core kernel on its MMAs gave up */
    GF_ESTATE = 7      /* inputs missing (e.g. gf_local before gf_set_sigma)        */
} gf_status;

/* Arithmetic of the (k, i w_n) point kernels.  Reductions over k and n, the
 * Matsubara tail and the mu search run in FP64 in every mode.
 *  GF_PREC_FP64  embedding, inverse and projections in FP64.
 *  GF_PREC_MIXED embedding and Gauss-Jordan inverse in single-word FP32
 *                (register tiles, windows up to 128 bands; wider windows use
 *                the GF_PREC_PAIR kernels), the Matsubara sums of G in FP64;
 *                the columns of G that G_loc and the adjoint consume
 *                (G P^+ and P G) get one step of iterative refinement with a
 *                residual in FP32 pairs.  Errors against FP64: about
 *                kappa(A) 2^-24 per G entry before refinement, which averages
 *                to ~1e-9 relative on N(mu); ~1e-11 on G_loc after it.
 *                N(mu) passes of windows up to 96 bands may run one to three
 *                warps per matrix, and the other passes of windows up to 40
 *                bands one warp per matrix with the CTA's refined projections
 *                (the autotuner's choice, the same arithmetic).  The environment
 *                variable GF_KERNEL restricts the candidates: f32r (register
 *                tiles), w32 (the warp kernels), or tc, which runs the N(mu)
 *                passes on the tcgen05 tensor cores (blocked elimination, TF32
 *                split operands): N within ~1e-7 of FP64.
 *  GF_PREC_PAIR  every matrix entry an FP32 pair (hi + lo) with error-free
 *                transformations on the FP32 pipes: ~1e-14 of FP64 results. */
typedef enum { GF_PREC_FP64 = 0, GF_PREC_MIXED = 1, GF_PREC_PAIR = 2 } gf_precision;
typedef enum { GF_C128 = 0, GF_C64 = 1 } gf_dtype;

typedef struct {
    int32_t n_systems;        /* >= 1: independent lattice problems in one context              */
    int32_t n_k;              /* total k-points over all systems                                 */
    const int32_t *nb;        /* host [n_k]: band-window size N_b(k) >= 1, or NULL: nb_uniform   */
    int32_t nb_uniform;       /* used when nb == NULL                                            */
    const int32_t *k_system;  /* host [n_k]: system of each k (non-decreasing), or NULL: all 0   */
    const int32_t *m_system;  /* host [n_systems]: correlated orbitals m >= 1 of each system      */
    int32_t n_iw;             /* positive Matsubara frequencies, >= 1                            */
    const double *beta;       /* host [n_systems]: inverse temperature > 0                       */
    const double *k_weight;   /* host [n_k]: w_k, or NULL: 1/N_k of the k's system               */
    int32_t precision;        /* gf_precision                                                    */
    int32_t input_dtype;      /* gf_dtype of the arrays given to gf_set_*                        */
    int32_t tail_order;       /* 1 or 2 (2 recommended)                                          */
    int32_t device;           /* CUDA device ordinal                                             */
    void *stream;             /* cudaStream_t to order all work on, or NULL (legacy default)     */
    int32_t flags;            /* GF_FLAG_* bits                                                  */
    const int32_t *system_dtype; /* host [n_systems]: gf_dtype of each system's blocks in the    */
                              /* arrays given to gf_set_*, or NULL: input_dtype for every system */
} gf_desc;

/* gf_desc.flags: replay the N(mu) evaluation (gf_occupation, each step of
 * gf_find_mu) as a CUDA graph.  The first evaluation runs normally (it sizes the
 * scratch and runs the autotuner), the second is captured on a library-owned
 * stream, later ones replay the graph with mu read from pinned memory at launch.
 * The library orders the replay after the context's stream and waits for it. */
#define GF_FLAG_GRAPH 1

/* gf_desc.flags: evaluate every (k, i w_n) point in the eigenbasis of H_k
 * (Woodbury identity): H_k = U diag(eps) U^+ is diagonalised once per
 * Hamiltonian upload (batched Jacobi kernel), after which a point costs
 * 3 N_b m^2 + O(m^3) complex multiply-adds instead of N_b^3.  Same results as
 * the direct inverse up to rounding; N_b <= 256.  With GF_PREC_MIXED or
 * GF_PREC_PAIR the band sums of g0, g1, g2 (the N_b m^2 part) run in FP32-pair
 * arithmetic and the m x m algebra in FP64.  With
 * GF_FLAG_GRAPH the eigen-decomposition runs outside the replayed graph, once
 * after each upload of H or P.  U^+ G U = D + D Pt^+ K Pt D with D = diag(1/(i w + mu - eps)),
 * Pt = P_k U, K = (I - Sigma Pt D Pt^+)^{-1} Sigma. */
#define GF_FLAG_LOWRANK 2

/* Create a context: validates the descriptor, copies it, selects the device
 * and allocates the device-side tables.  *out is NULL on failure.
 * Errors: GF_EINVAL, GF_ENOMEM, GF_ECUDA. */
gf_status gf_create(gf_ctx **out, const gf_desc *desc);

/* Release every device and host resource of the context (NULL is a no-op). */
gf_status gf_destroy(gf_ctx *ctx);

/* H_k for all k (Sec. 3.1, Eq. H_LDA in the band window): packed per k, an
 * N_b(k) x N_b(k) Hermitian block (is_diagonal = 0) or the N_b(k) diagonal
 * entries E_nk (is_diagonal != 0, stored as complex with zero imaginary part).
 * Hermiticity is the caller's contract and is not checked.
 * Errors: GF_EINVAL (NULL), GF_ECUDA. */
gf_status gf_set_hamiltonian(gf_ctx *ctx, const void *h_ptr, int32_t is_diagonal);

/* P_k = S^k_{alpha n} = <alpha_k | phi_nk> (Sec. 3.1, Eq. S_norm): packed per k,
 * an m(system) x N_b(k) block.  Orthonormal rows are not assumed.
 * Errors: GF_EINVAL, GF_ECUDA. */
gf_status gf_set_projectors(gf_ctx *ctx, const void *p_ptr);

/* Sigma(i w_n) (Sec. 3.2.4): packed per system [n_iw][m][m], and Sigma(inf):
 * packed per system [m][m] (Hermitian; the double-counting shift -V_DC is to be
 * folded in by the caller, as H_ps of Eq. pseudo_H_k does).
 * Errors: GF_EINVAL, GF_ECUDA. */
gf_status gf_set_sigma(gf_ctx *ctx, const void *sigma_iw_ptr, const void *sigma_inf_ptr);

/* G_loc(i w_n) = sum_k w_k P_k G P_k^+ (Eq. dmftloop2) at mu[s] (host [n_systems]).
 * Output: packed per system [n_iw][m][m] complex128, host or device.
 * Errors: GF_ESTATE (inputs missing), GF_ESINGULAR, GF_EINVAL, GF_ECUDA. */
gf_status gf_local(gf_ctx *ctx, const double *mu, void *gloc_out_ptr);

/* N(mu) = sum_k w_k Tr rho_k (Eq. fix_mu) and dN/dmu per system, to host
 * arrays [n_systems] (dn_dmu_out may be NULL).
 * Errors: GF_ESTATE, GF_ESINGULAR, GF_EINVAL, GF_ECUDA. */
gf_status gf_occupation(gf_ctx *ctx, const double *mu, double *n_out, double *dn_dmu_out);

/* Chemical potential of every system with |N(mu) - n_target[s]| <= tol
 * (Eq. fix_mu), by safeguarded Newton steps on N(mu) with a bisection bracket.
 * mu_inout [n_systems] holds the start values and receives the result;
 * iters_out (may be NULL) receives the number of N(mu) evaluations.
 * Errors: GF_ENOTCONV (mu_inout then holds the best iterate), GF_ESTATE,
 * GF_ESINGULAR, GF_EINVAL, GF_ECUDA. */
gf_status gf_find_mu(gf_ctx *ctx, const double *n_target, double tol, int32_t max_iter,
                     double *mu_inout, int32_t *iters_out);

/* rho_k (Eq. rho_LDA+DMFT) for every k, packed per k as N_b(k) x N_b(k)
 * complex128 (host or device), and n_corr = sum_k w_k Tr(P_k rho_k P_k^+)
 * (Eq. nf_LDA+DMFT) per system to host [n_systems] (may be NULL).
 * rho_out_ptr may be NULL to get n_corr only.
 * Errors: GF_ESTATE, GF_ESINGULAR, GF_EINVAL, GF_ECUDA. */
gf_status gf_density_matrix(gf_ctx *ctx, const double *mu, void *rho_out_ptr, double *n_corr_out);

/* One fused pass over every (k, i w_n) point at mu[s]: any subset of G_loc
 * (as gf_local), rho_k (as gf_density_matrix), N and dN/dmu (as gf_occupation)
 * and n_corr; NULL outputs are not computed.  Each G(k, i w_n) is formed and
 * inverted once for all requested outputs.
 * Errors: GF_ESTATE, GF_ESINGULAR, GF_EINVAL (all outputs NULL), GF_ECUDA. */
gf_status gf_evaluate(gf_ctx *ctx, const double *mu, void *gloc_out_ptr, void *rho_out_ptr,
                      double *n_out, double *dn_dmu_out, double *n_corr_out);

/* Vector-Jacobian product (not in the paper; derived from Eq. dmftloop1 with
 * dG = G P^+ dSigma P G and dG/dmu = -G^2).  For a real loss L with
 * dL = Re<gloc_bar, dG_loc> + n_bar . dN, and the convention
 * grad z = dL/dRe z + i dL/dIm z:
 *   sigma_bar(w_n) = sum_k w_k [A_k^+ gloc_bar(w_n) A_k^+ + n_bar (2/beta) B_k^+],
 *   mu_bar         = n_bar dN/dmu - sum_n sum_k w_k Re<gloc_bar(w_n), B_k>,
 * with A_k = P_k G P_k^+ and B_k = P_k G G P_k^+.
 * gloc_bar_ptr: packed per system [n_iw][m][m] complex128 or NULL (= 0);
 * n_bar: host [n_systems] or NULL (= 0).  sigma_bar_out_ptr: packed like
 * Sigma(i w_n), complex128, host or device.  mu_bar_out: host [n_systems].
 * Errors: GF_ESTATE, GF_ESINGULAR, GF_EINVAL, GF_ECUDA. */
gf_status gf_backward(gf_ctx *ctx, const double *mu, const void *gloc_bar_ptr, const double *n_bar,
                      void *sigma_bar_out_ptr, double *mu_bar_out);

/* N(mu) and dN/dmu of one system with a uniform band window, without any
 * device allocation.  The paper has no counterpart: this is a library
 * service for callers that cannot call cudaMalloc, such as code running
 * inside another framework's memory pool or allocator hooks, plugins that may
 * not grow the device footprint after start-up, or hot paths where allocation
 * is forbidden.  It computes what gf_occupation computes for a context made
 * of these sizes, with the same point kernel.
 *
 * Inputs are device pointers of the current device, complex128: h_dev
 * [n_k][nb][nb], p_dev [n_k][m][nb], sigma_dev [n_iw][m][m], sigma_inf_dev
 * [m][m]; k-weights are 1/n_k.  stream: cudaStream_t or NULL.  Results go to
 * the host: *n_out and, if not NULL, *dn_dmu_out; the call returns after the
 * stream has drained.
 *
 * Scratch: a file-scope device array of 4 MiB that every GPU loading the
 * library holds until the process exits.  The problem must fit in it:
 * about 32 bytes per (k, frequency chunk) item plus 56 bytes per k-point
 * (n_k = 1000 with 1024 frequencies needs about 0.5 MiB); larger problems,
 * and windows whose matrix does not fit in shared memory, return GF_EINVAL.
 * Each call looks up the array's address on the current device.  Every call
 * shares the one array and overwrites it, so calls whose work overlaps on the
 * GPU (other streams, other host threads) race: serialise them.
 * Errors (message in gf_last_error(NULL)): GF_EINVAL, GF_ESINGULAR, GF_ECUDA. */
gf_status gf_occupation_static(const void *h_dev, const void *p_dev, const void *sigma_dev,
                               const void *sigma_inf_dev, int32_t n_k, int32_t nb, int32_t m,
                               int32_t n_iw, double beta, double mu, int32_t tail_order,
                               void *stream, double *n_out, double *dn_dmu_out);

/* ---- Pole form of Sigma: the pseudo-Hamiltonian path (Sec. 3.3) ----------
 * When Sigma has the pole form of Sec. 3.2.4 (Eq. se_pole),
 *   Sigma(i w) = Sigma_inf + sum_i V_i^+ V_i / (i w - p_i),  V_i a 1 x m row,
 * the band block of the resolvent of the pseudo-Hamiltonian (Eq. pseudo_H_k)
 *   H_ps = [[H_k + P_k^+ Sigma_inf P_k, W^+], [W, diag(p_i + mu)]],  W_i = V_i P_k,
 * equals G(k, i w_n) of Eq. dmftloop1 at every frequency, and rho_k, N(mu),
 * n_corr and G_loc follow from its eigenpairs in closed form (Eqs.
 * rho_LDA+DMFT_componet_final, fix_mu; no Matsubara truncation and no tail).
 * The pole energies enter shifted by mu because Sigma is a function of i w
 * (the reading the Matsubara path uses too), so each mu diagonalises H_ps
 * again: one (N_b + n_poles)-square Hermitian eigenproblem per k, solved by
 * the library's batched Jacobi kernel (N_b + n_poles <= 256). */

/* Pole form of Sigma per system: n_poles [n_systems] (host), pole energies
 * p [sum_s n_poles[s]] (real, eV, host or device), pole vectors
 * V [sum_s n_poles[s] * m_s] (complex of the context's input dtype, row i of
 * system s holds V_i), Sigma_inf [sum_s m_s^2] (complex, Hermitian).  The
 * library copies them; the Matsubara-path Sigma of gf_set_sigma is untouched.
 * Errors: GF_EINVAL (NULL pointers, negative n_poles, a non-finite pole,
 * N_b + n_poles > 256, m > 32), GF_ENOMEM, GF_ECUDA. */
gf_status gf_set_sigma_poles(gf_ctx *ctx, const int32_t *n_poles, const double *poles_ptr,
                             const void *v_ptr, const void *sigma_inf_ptr);

/* N(mu) = sum_k w_k sum_l |Psi_b,l|^2 n_F(E_l - mu) and its exact derivative
 * dN/dmu per system (host arrays [n_systems]; dn_dmu_out may be NULL), from the
 * eigenpairs (E_l, Psi_l) of H_ps(mu); Psi_b,l is the band block of Psi_l.
 * Errors: GF_ESTATE (H, P or the poles missing), GF_ENOTCONV (Jacobi did not
 * converge in 40 sweeps), GF_EINVAL, GF_ECUDA. */
gf_status gf_pole_occupation(gf_ctx *ctx, const double *mu, double *n_out, double *dn_dmu_out);

/* mu per system with |N(mu) - n_target[s]| <= tol on the pole-path N(mu), by
 * the same safeguarded Newton iteration as gf_find_mu.
 * Errors: as gf_find_mu and gf_pole_occupation. */
gf_status gf_pole_find_mu(gf_ctx *ctx, const double *n_target, double tol, int32_t max_iter,
                          double *mu_inout, int32_t *iters_out);

/* rho_k = Psi_b diag(n_F(E - mu)) Psi_b^+ packed per k like gf_density_matrix
 * (host or device, may be NULL) and n_corr = sum_k w_k Tr(P_k rho_k P_k^+) per
 * system to host [n_systems] (may be NULL).
 * Errors: as gf_pole_occupation. */
gf_status gf_pole_density_matrix(gf_ctx *ctx, const double *mu, void *rho_out_ptr,
                                 double *n_corr_out);

/* G_loc(i w_n) = sum_k w_k sum_l phi_l phi_l^+ / (i w_n + mu - E_l), phi_l =
 * P_k Psi_b,l, on the context's n_iw Matsubara frequencies, packed like
 * gf_local's output (complex128, host or device).
 * Errors: as gf_pole_occupation. */
gf_status gf_pole_local(gf_ctx *ctx, const double *mu, void *gloc_out_ptr);

/* Density of states on the real axis from the pseudo-Hamiltonian eigenpairs
 * (Eqs. DOS and PDOS), broadened by a Lorentzian of half width eta > 0:
 *   D(e) = -(1/pi) Im sum_k w_k sum_l |Psi_b,l|^2 / (e + mu - E_l + i eta),
 *   D_alpha(e) = -(1/pi) Im sum_k w_k sum_l |(P_k Psi_b,l)_alpha|^2 / (same).
 * eps [n_eps] energies relative to mu (host or device); dos_out host or device
 * [n_systems][n_eps]; pdos_out (may be NULL) host or device, per system
 * [n_eps][m_s], systems one after the other.
 * Errors: as gf_pole_occupation, GF_EINVAL (n_eps < 1, eta <= 0). */
gf_status gf_pole_spectral(gf_ctx *ctx, const double *mu, int32_t n_eps, const double *eps,
                           double eta, double *dos_out, double *pdos_out);

/* Energy terms of Sec. 3.4 from the pseudo-Hamiltonian eigenpairs, per system
 * to host [n_systems] (either pointer may be NULL):
 *   h_ks = sum_k w_k Tr(H_k rho_k)                              (Eq. H_KS)
 *   e_ps = sum_k w_k sum_l (E_l - mu) |Psi_b,l|^2 n_F(E_l - mu)
 * so that <H_U> = (e_ps - h_ks + <V_DC>) / 2 (Eq. H_U_energy).
 * Errors: as gf_pole_occupation. */
gf_status gf_pole_energy(gf_ctx *ctx, const double *mu, double *h_ks_out, double *e_ps_out);

/* Batched Hermitian eigensolver (cyclic Jacobi, the kernel of the pole path),
 * stateless: a [n_mat][n][n] complex128 on the device (its Hermitian part
 * (A + A^+)/2 is used) -> eigenvalues w [n_mat][n] ascending and eigenvectors
 * v [n_mat][n][n] (column l of each matrix is the vector of w[l]), both device
 * arrays.  1 <= n <= 256; at most max_sweeps sweeps.  Enqueued on stream
 * (NULL = legacy default) and synchronised before return; scratch comes from
 * the stream-ordered allocator.  The paper needs it inside the pseudo-
 * Hamiltonian method of Sec. 3.3; this entry exposes it on its own.
 * Errors (message in gf_last_error(NULL)): GF_EINVAL (sizes, host pointers),
 * GF_ENOTCONV, GF_ENOMEM, GF_ECUDA. */
gf_status gf_heev_batched(const void *a_dev, int32_t n_mat, int32_t n, int32_t max_sweeps,
                          double *w_dev, void *v_dev, void *stream);

/* ---- Around the lattice sums: projectors and the DMFT step ----------------- */

/* Orthonormal projectors (Eqs. 6 and 7): from raw projections W_k (packed like
 * P, m x N_b(k) per k, input dtype, host or device) the library computes
 * P_k = O_k^{-1/2} W_k with the overlap O_k = W_k W_k^+ (m x m), by one
 * Hermitian eigenproblem of O_k per k, and makes P_k the context's projectors
 * (as gf_set_projectors would).  p_out_ptr (may be NULL) receives P_k as
 * complex128.  m <= 32.
 * Errors: GF_ESINGULAR (an overlap eigenvalue <= 1e-12 of the largest: the
 * projections of a k-point are linearly dependent), GF_EINVAL, GF_ECUDA. */
gf_status gf_set_projectors_lowdin(gf_ctx *ctx, const void *w_ptr, void *p_out_ptr);

/* Impurity levels (Eq. E^imp): E_imp = sum_k w_k P_k H_k P_k^+ - V_DC I per
 * system, [sys][m][m] complex128 (host or device).  v_dc: host [n_systems]
 * double-counting potentials V_DC (Eq. V_DC_component), or NULL for 0.
 * Errors: GF_ESTATE (H or P missing), GF_EINVAL, GF_ECUDA. */
gf_status gf_impurity_levels(gf_ctx *ctx, const double *v_dc, void *e_imp_out_ptr);

/* Hybridization function of the DMFT self-consistency step (Eq. dmftloop2):
 *   Delta(i w_n) = (i w_n + mu) I - E_imp - Sigma(i w_n) - G_loc(i w_n)^{-1}
 * for every system and frequency, from G_loc (complex128, packed like
 * gf_local's output, host or device; e.g. that output), the context's Sigma
 * (gf_set_sigma) and E_imp with v_dc as in gf_impurity_levels.  delta_out_ptr:
 * complex128 packed like Sigma (host or device).  m <= 32.
 * Errors: GF_ESTATE (Sigma, H or P missing), GF_ESINGULAR (G_loc singular at a
 * frequency), GF_EINVAL, GF_ECUDA. */
gf_status gf_hybridization(gf_ctx *ctx, const double *mu, const void *gloc_ptr, const double *v_dc,
                           void *delta_out_ptr);

/* Double counting of Sec. 3.2.3 (host arithmetic, no context): for interaction
 * U, Hund's coupling J, orbital quantum number l (M = 2l + 1) and occupation n
 * of the correlated shell,
 *   U_bar = (U + 2(M-1)(U-2J) - (M-1)J) / (2M-1)      (Eq. U_eff)
 *   V_DC  = U_bar (n - 1/2)                           (Eq. V_DC_component)
 *   E_DC  = U_bar n (n - 1) / 2                        (Eq. E_DC)
 * Any output pointer may be NULL.  Errors: GF_EINVAL (non-finite input, l < 0). */
gf_status gf_double_counting(double U, double J, int32_t l, double n, double *u_bar_out,
                             double *v_dc_out, double *e_dc_out);

/* Message of the last failed call on this context ("" if none).  Owned by the
 * context, valid until the next call on it. */
const char *gf_last_error(const gf_ctx *ctx);

/* How the library configured its kernels for this context (e.g. which
 * mixed-precision kernel the autotuner kept and the timings it compared), as a
 * context-owned string ("" before the first compute call). */
const char *gf_tuning_log(const gf_ctx *ctx);

/* Counters of the last compute call (any pointer may be NULL): kernel launches
 * of this library, (k, i w_n) points evaluated, the summed duration of the
 * point-kernel launches in milliseconds (CUDA events recorded on the context's
 * stream around each launch), and their algorithmic floating-point operations
 * (8 per complex multiply-add: N_b^3 for the inverse, m^2 N_b + m N_b^2 for the
 * embedding, plus the epilogue's projections and traces). */
gf_status gf_last_stats(const gf_ctx *ctx, int64_t *kernel_launches, int64_t *points,
                        double *point_kernel_ms, double *point_flops);

#ifdef __cplusplus
}
#endif

#endif /* GF_H */

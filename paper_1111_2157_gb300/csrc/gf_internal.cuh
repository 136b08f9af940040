// Internal declarations shared by the CUDA translation units of libgf.
// Nothing here is part of the C-ABI (include/gf.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <new>
#include <stdexcept>

#include "gf.h"

namespace gf {

constexpr int kThreads = 256;          // threads per CTA of every point kernel
constexpr int kFlagSingular = 1;       // status bit: zero or non-finite pivot
constexpr int kFlagTimeout = 2;        // status bit: a bounded wait on the tensor cores gave up
constexpr int kMaxKGroup = 16;         // k-points per k-group item (modes with a k-reduction)

// Work modes of the point kernels (bit set).
enum Mode : int {
  kOcc = 1,    // Re Tr sum_n G and Re Tr sum_n G^2 per (k, chunk): N(mu), dN/dmu
  kRho = 2,    // S_k = sum_n G(k, i w_n) per (k, chunk): rho_k
  kGloc = 4,   // w_k P_k G P_k^+ per (k, n): G_loc after the k-reduction
  kAdj = 8,    // w_k [A^+ Gbar A^+ + nbar (2/beta) B^+] per (k, n) and mu_bar partials
};

struct KInfo {          // one k-point
  int nb;               // band-window size N_b(k)
  int sys;              // system index
  int64_t offH;         // offset of the N_b x N_b block in H / E_inf / rho (complex elements)
  int64_t offP;         // offset of the m x N_b block in P (complex elements)
  double w;             // k weight w_k
};

struct SInfo {          // one system
  int m;                // correlated orbitals
  int k0, k1;           // its k-points are [k0, k1)
  int pad;
  double beta;
  double tailc;         // (2/beta) sum_{n<n_iw} 1/w_n^2 - beta/4 for tail_order 2, else 0
  int64_t offSig;       // offset of [n_iw][m][m] in Sigma / G_loc / Sigma_bar (complex elements)
  int64_t offSinf;      // offset of [m][m] in Sigma_inf (complex elements)
};

// One unit of work: frequencies [n0, n1) of nk k-points.  Modes with a k-reduction (kGloc,
// kAdj) take the k-points kperm[k .. k+nk) of k-group g, whose contributions the CTA sums in
// k order into one slot per (group, frequency); the other modes take the single k-point k
// (nk = 1, no kperm).
struct Item {
  int k, n0, n1, chunk, nk, g;
};

struct PointParams {
  // inputs (device, complex128 interleaved)
  const double2* H;
  const double2* P;
  const double2* Sig;
  const KInfo* kinfo;
  const SInfo* sinfo;
  const Item* items;
  int n_items;
  int n_chunks;         // chunks per k (occ / mu_bar partial layout [k][chunk])
  int* queue;           // work counter, zero before launch
  const double* mu;     // [n_sys]
  int mode;
  int nmat;             // df64 kernel: frequencies processed together per CTA (1..4)
  int nbmax, mmax;
  int a_in_smem;        // 1: the N_b x N_b matrix lives in shared memory
  double2* a_scratch;   // else: per-CTA slices of a_stride elements in global memory
  int64_t a_stride;
  // FP32-pair copies of H, P, Sigma and Gbar for the df64 kernel: {re.hi, re.lo, im.hi, im.lo}
  const float4* Hd;
  const float4* Pd;
  const float4* Sd;
  const float4* Gbd;
  // single-word FP32 copies of H, P and Sigma for the f32r kernel
  const float2* Hs;
  const float2* Ps;
  const float2* Ss;
  // outputs
  double* occ_part;     // [n_k][n_chunks][2]
  double2* rho_part;    // [n_chunks][sum_k N_b^2]
  int64_t rho_chunk_stride;
  double2* gq;          // [g - gb0][n][mmax^2]: k-group sums of w_k P G P^+ (or the adjoint's)
  int gb0;              // first k-group of the batch
  const int* kperm;     // k-points of the k-groups (group items), or null (single-k items)
  int n_iw;
  // adjoint
  const double2* gbar;  // [sum_s n_iw m_s^2] or null
  const double* nbar;   // [n_sys] device, or null
  double* mubar_part;   // [n_k][n_chunks]
  int* status;
  int tc_skip_mma;      // tensor-core kernel, failure-detection tests only: issue no MMA, so
                        // the bounded wait for it runs out and the kernel reports kFlagTimeout
};

struct PInfo {          // pole form of one system's Sigma
  int np;               // number of poles
  int pad;
  int64_t offp;         // offset of its poles in the pole-energy array
  int64_t offV;         // offset of its [np][m] pole vectors (complex elements)
};

struct PoleParams {
  const double2* H;
  const double2* P;
  const double2* Sinf;  // [sys][m][m], offsets SInfo::offSinf
  const double* poles;
  const double2* Vp;
  const KInfo* kinfo;
  const SInfo* sinfo;
  const PInfo* pinfo;
  const double* mu;     // [n_sys]
  int n_k, n_iw, mode, max_sweeps;
  int in_smem;          // 1: H_ps and its eigenvectors in shared memory
  double2* ws;          // else per-CTA slices of ws_stride elements
  int64_t ws_stride;
  double* kN;           // [n_k] N_k
  double* kdN;          // [n_k] dN_k/dmu
  double* kNc;          // [n_k] n_corr,k
  double2* rho;         // packed like H
  double* eout;         // eigenvalues per k at eoff[k]
  double2* phiout;      // P Psi_b per k, [m][N_b + np] at phioff[k]
  const int64_t* eoff;
  const int64_t* phioff;
  double2* gloc;        // [sys][n_iw][m][m] at SInfo::offSig
  double* wbout;        // band weights |Psi_b,l|^2 per k at eoff[k] (kGloc), or null
  double* kHks;         // [n_k] Re Tr(H_k rho_k) (kRho), or null
  double* kEps;         // [n_k] sum_l (E_l - mu) |Psi_b,l|^2 n_F (kRho), or null
  // warm start of the mu search: eigenpairs of the previous evaluation
  double2* vstore;      // eigenvectors per k, [n][n] at voff[k] (row i, column l), or null
  double* estore;       // eigenvalues per k at eoff[k]
  const int64_t* voff;
  const double* mu_prev;  // [n_sys] mu of the stored eigenpairs
  int warm;             // 1: start Jacobi from the stored eigenpairs
  int save_v;           // 1: store this evaluation's eigenpairs
  int* status;
};

__host__ __device__ inline int imax(int a, int b) { return a > b ? a : b; }

// k-point q of an item (see Item)
__device__ __forceinline__ int item_k(const Item& it, const int* kperm, int q) {
  return kperm ? kperm[it.k + q] : it.k + q;
}
// slot of a k-group sum: the first k-point of the group writes, the later ones add (in k order).
// The slot is stored and reloaded with an L2 evict-last policy: a CTA revisits its group's
// slots one chunk of frequencies later, and the policy keeps them in L2 until then instead
// of writing each visit back to HBM.
__device__ __forceinline__ void gq_put(double2* out, int q, double2 v) {
  uint64_t pol;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  if (q) {
    double2 o;
    asm volatile("ld.global.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;"
                 : "=d"(o.x), "=d"(o.y)
                 : "l"(out), "l"(pol));
    v.x += o.x;
    v.y += o.y;
  }
  asm volatile("st.global.L2::cache_hint.v2.f64 [%0], {%1, %2}, %3;" ::"l"(out), "d"(v.x), "d"(v.y), "l"(pol)
               : "memory");
}

// Thread t's share (of nthr threads) of Re Tr H_k + Re Tr(Sigma_inf P_k P_k^+), the trace
// of the first-moment matrix H_k + P_k^+ Sigma_inf P_k that the tail needs; summing the
// shares over the threads gives the trace.  (P P^+)_ba = sum_i P_bi conj(P_ai).  Shared by
// the context path (k_einf) and the allocation-free path so that both compute it alike.
__device__ inline double trhe_partial(const double2* __restrict__ Hk, const double2* __restrict__ Pk,
                                      const double2* __restrict__ S, int nb, int m, int t, int nthr) {
  double v = 0.0;
  for (int i = t; i < nb; i += nthr) v += Hk[(int64_t)i * nb + i].x;
  for (int e = t; e < m * m; e += nthr) {
    const int a = e / m, b = e - a * m;
    double re = 0.0, im = 0.0;
    for (int i = 0; i < nb; ++i) {
      const double2 x = Pk[b * nb + i], y = Pk[a * nb + i];
      re = fma(x.x, y.x, fma(x.y, y.y, re));
      im = fma(x.y, y.x, fma(-x.x, y.y, im));
    }
    const double2 sv = S[a * m + b];
    v = fma(sv.x, re, fma(-sv.y, im, v));
  }
  return v;
}

// Eigenbasis data of the low-rank path: H_k = U diag(eps) U^+, Pt = P_k U.
struct LowRank {
  const double* eps;     // [sum_k N_b] at offD[k]
  const int64_t* offD;
  const double2* Pt;     // [m][N_b] per k at KInfo::offP
  int t_in_smem;         // 1: the pair table Pt_ab conj(Pt_cb) of an item is kept in shared memory
  int pair_sums;         // 1: the band sums of g0, g1, g2 in FP32-pair arithmetic (mixed precision)
};

// Shared-memory layout of k_point_lr (16-byte complex elements).  offT: the
// pair table T[p][b] = Pt_ab conj(Pt_cb), p over the pairs a <= c (m(m+1)/2).
struct LRLayout {
  int offPt, offD, offS, offG, offAug, offC, offC2, offX, offCol, offU, offT, offPtd, offDd;
  size_t bytes;
};

__host__ __device__ inline LRLayout make_lr_layout(int nbmax, int mmax, int mode, int t_in_smem,
                                                   int pair_sums) {
  LRLayout L;
  const int mm = mmax * mmax;
  int o = 0;
  L.offPt = o; o += mmax * nbmax;
  L.offD = o; o += 3 * nbmax;
  L.offS = o; o += mm;
  L.offG = o; o += 3 * mm;
  L.offAug = o; o += 2 * mm;
  L.offC = o; o += mm;
  L.offC2 = o; o += mm;
  L.offX = o; o += imax((mode & kRho) ? mmax * nbmax : 0, (mode & kAdj) ? 4 * mm : 0);
  L.offCol = o; o += 2 * mmax;
  L.offU = o; o += 2 * mmax;
  L.offT = o; o += t_in_smem ? (mmax * (mmax + 1) / 2) * nbmax : 0;
  L.offPtd = o; o += pair_sums ? mmax * nbmax : 0;  // FP32-pair copies of Pt and of d, d^2, d^3
  L.offDd = o; o += pair_sums ? 3 * nbmax : 0;
  L.bytes = (size_t)o * 16;
  return L;
}

size_t point_lr_smem(int nbmax, int mmax, int mode, int t_in_smem, int pair_sums);
int point_lr_blocks_per_sm(size_t smem, int pair_sums);
cudaError_t launch_point_lr(const PointParams& p, const LowRank& lr, int grid, size_t smem,
                            cudaStream_t s);
cudaError_t launch_lr_rotate(const KInfo* kinfo, int n_k, const double2* U, double2* rho_part,
                             int64_t stride, int n_chunks, double2* T, cudaStream_t s);
// Eigen-decomposition of every H_k (Jacobi): eps [offD], U [offH], Pt = P U [offP].
cudaError_t launch_lr_setup(const double2* H, const double2* P, const KInfo* kinfo,
                            const SInfo* sinfo, const int64_t* offD, int n_k, int nbmax,
                            double* eps, double2* U, double2* Pt, double2* ws, int grid,
                            int in_smem, int* status, cudaStream_t s);

// DMFT self-consistency step: E_imp = sum_k w_k P H P^+ - V_DC (part: [n_k][mmax^2]
// scratch; out: [sys][m][m] at SInfo::offSinf) and Delta(i w_n) (packed like Sigma).
cudaError_t launch_eimp(const KInfo* kinfo, const SInfo* sinfo, int n_k, int n_sys, const double2* H,
                        const double2* P, int nbmax, int mmax, double2* part, const double* v_dc,
                        double2* out, cudaStream_t s);
cudaError_t launch_hybridization(const SInfo* sinfo, int n_sys, int n_iw, int mmax, const double* mu,
                                 const double2* eimp, const double2* Sig, const double2* gloc,
                                 double2* delta, int* status, cudaStream_t s);
// Lowdin-orthonormal projectors P_k = (W_k W_k^+)^{-1/2} W_k (packed like P).
cudaError_t launch_lowdin(const KInfo* kinfo, const SInfo* sinfo, int n_k, int mmax,
                          const double2* Wraw, double2* Pout, int* status, cudaStream_t s);

// Batched Hermitian eigensolver (cyclic Jacobi) and the pole path.
size_t heev_smem(int n);
size_t heev_ws_elems(int n);
int heev_max_n();
cudaError_t launch_heev_batched(const double2* A, int n_mat, int n, int max_sweeps, double* w,
                                double2* V, double2* gws, int grid, int in_smem, int* status,
                                cudaStream_t s);
cudaError_t launch_pole_eig(const PoleParams& p, int grid, size_t smem, cudaStream_t s);
// G_loc from the eigenpairs, k split n_split ways into part [n_split][tot] and
// summed in split order into p.gloc.
int pole_gloc_splits(int n_sys, int n_iw, int sm_count, int mmax);
cudaError_t launch_pole_gloc(const PoleParams& p, int n_sys, int mmax, int n_split, double2* part,
                             int64_t tot, cudaStream_t s);
cudaError_t launch_pole_dos(const PoleParams& p, int n_sys, const double* eps_grid, int n_eps,
                            double eta, const int64_t* pdos_off, double* dos, double* pdos,
                            cudaStream_t s);

// Shared-memory layout of the point kernels, in 16-byte complex elements (a
// complex double or a complex FP32 pair): the N_b x N_b matrix (odd leading
// dimension), P_k, T = Sigma P_k / Y = G P^+ / Gbar A^+, Z = P G (adjoint),
// Sigma(i w_n) / Gbar, A_k and B_k (adjoint), the pivot column and row, then the
// pivot and column-permutation index arrays.
struct Layout {
  int offA, offP, offT, offZ, offS, offQa, offQb, offCol, offU;
  int n2;        // 16-byte elements before the int arrays
  size_t bytes;
};


__host__ __device__ inline Layout make_layout(int nbmax, int mmax, int mode, int a_in_smem) {
  Layout L;
  const int ld = nbmax | 1;
  int o = 0;
  L.offA = o; o += a_in_smem ? nbmax * ld : 0;
  L.offP = o; o += mmax * nbmax;
  L.offT = o; o += imax(mmax * nbmax, mmax * mmax);
  L.offZ = o; o += (mode & kAdj) ? mmax * nbmax : 0;
  L.offS = o; o += mmax * mmax;
  L.offQa = o; o += (mode & kAdj) ? mmax * mmax : 0;
  L.offQb = o; o += (mode & kAdj) ? mmax * mmax : 0;
  L.offCol = o; o += nbmax;
  L.offU = o; o += nbmax;
  L.n2 = o;
  L.bytes = (size_t)o * 16 + 2 * (size_t)nbmax * sizeof(int);
  return L;
}

// Shared-memory footprint (bytes) of k_point_fp64 for the given sizes and mode.
size_t point_fp64_smem(int nbmax, int mmax, int mode, int a_in_smem);

cudaError_t launch_point_fp64(const PointParams& p, int grid, size_t smem, cudaStream_t s);
int point_fp64_blocks_per_sm(size_t smem);
cudaError_t launch_point_df64(const PointParams& p, int grid, size_t smem, cudaStream_t s);
int point_df64_blocks_per_sm(size_t smem);
// Register-resident FP32-pair kernel (windows up to 96 bands): tile shape for a
// maximum window (-1 if none), its thread count, shared memory and occupancy.
int df64r_shape(int nbmax);
int df64r_num_shapes();
int df64r_tile(int shape, int which);  // RA (which = 0) or RB (which = 1) of a shape
bool df64r_shape_fits(int shape, int nbmax);
int df64r_threads(int shape, int nbmax);
size_t point_df64r_smem(int nbmax, int mmax, int mode);
int point_df64r_blocks_per_sm(int shape, int threads, size_t smem);
cudaError_t launch_point_df64r(int shape, const PointParams& p, int grid, int threads, size_t smem,
                               cudaStream_t s);
// Mixed-precision register-resident FP32 kernel (gf_f32r.cu): tile shapes, the
// window class each serves, thread count, shared memory and occupancy.
int f32r_num_shapes();
int f32r_tile(int shape, int which);  // RA (which = 0) or RB (which = 1)
int f32r_nmax(int shape);
bool f32r_shape_fits(int shape, int nbmax);
int f32r_threads(int shape, int nbmax);
size_t point_f32r_smem(int nbmax, int mmax, int mode);
int point_f32r_blocks_per_sm(int shape, int threads, size_t smem);
// ... and its fused passes for windows up to 40 bands with one warp per matrix: each warp
// inverts one frequency, the CTA runs the refined projections (gf_f32r.cu).
int f32w_nmax(int nbmax);
int f32w_threads();
size_t point_f32w_smem(int nbmax, int mmax, int mode);
int point_f32w_blocks_per_sm(int nbmax, size_t smem);
cudaError_t launch_point_f32w(int nbmax, const PointParams& p, int grid, size_t smem, cudaStream_t s);

// Mixed-precision N(mu) kernel for windows up to 40 bands (gf_w32.cu): one warp per
// matrix, the matrix in registers.
int w32_nmax(int nbmax);
int w32_threads();
size_t point_w32_smem(int nbmax, int mmax);
int point_w32_blocks_per_sm(int nbmax, size_t smem);
cudaError_t launch_point_w32(int nbmax, const PointParams& p, int grid, size_t smem, cudaStream_t s);
// ... and windows of 41 to 96 bands: 2 or 3 warps per matrix, one row per lane.
int wm_nmax(int nbmax);
int wm_threads(int nbmax);
size_t point_wm_smem(int nbmax, int mmax);
int point_wm_blocks_per_sm(int nbmax, size_t smem);
cudaError_t launch_point_wm(int nbmax, const PointParams& p, int grid, size_t smem, cudaStream_t s);

// Mixed-precision N(mu) kernel on the tcgen05 tensor cores (gf_tc.cu): ng matrix
// groups of 128 threads per CTA, windows up to 128 bands.
bool tc_fits(int nbmax, int ng);
size_t point_tc_smem(int nbmax, int mmax, int ng);
int point_tc_blocks_per_sm(int nbmax, int ng, size_t smem);
cudaError_t launch_point_tc(int ng, const PointParams& p, int grid, size_t smem, cudaStream_t s);
cudaError_t launch_point_f32r(int shape, const PointParams& p, int grid, int threads, size_t smem,
                              cudaStream_t s);
// out[i] = complex FP32 rounding of in[i], for n complex numbers
cudaError_t launch_round_f32(const double2* in, float2* out, int64_t n, cudaStream_t s);
// Shared memory of k_point_df64 with nmat matrices (frequencies) per CTA step.
size_t point_df64_smem(int nbmax, int mmax, int mode, int a_in_smem, int nmat);
// out[i] = FP32 pair (hi, lo) of in[i], hi = RN(x), lo = RN(x - hi), for n complex numbers
cudaError_t launch_split_df64(const double2* in, float4* out, int64_t n, cudaStream_t s);
cudaError_t launch_occ_finalize(const KInfo* kinfo, const SInfo* sinfo, const double* trHE,
                                const double* mu, const double* occ_part, int n_chunks, int n_k,
                                double* kN, double* kdN, cudaStream_t s);
cudaError_t launch_sys_reduce(const KInfo* kinfo, const SInfo* sinfo, int n_sys, const double* a,
                              const double* b, double* out, cudaStream_t s);
cudaError_t launch_rho_finalize(const KInfo* kinfo, const SInfo* sinfo, const double2* H,
                                const double2* Einf, const double2* P, const double* mu,
                                const double2* rho_part, int64_t rho_chunk_stride, int n_chunks,
                                int n_k, double2* rho_out, double* kN, double* kNc, cudaStream_t s);
// acc[s] (+)= sum over the k-groups g of system s in [gb0, gb1), in increasing g, of gq[g - gb0];
// sys_g0 / sys_g1: [n_sys] first and end group of each system.
cudaError_t launch_gq_reduce(const SInfo* sinfo, int n_sys, int max_mm_total, const int* sys_g0,
                             const int* sys_g1, const double2* gq, int gb0, int gb1, int n_iw,
                             int mmax, int first, double2* acc, cudaStream_t s);
cudaError_t launch_einf(const KInfo* kinfo, const SInfo* sinfo, const double2* H, const double2* P,
                        const double2* Sinf, int n_k, double2* Einf, double* trHE, cudaStream_t s);
cudaError_t launch_upcast(const float2* in, double2* out, int64_t n, cudaStream_t s);
cudaError_t launch_diag_to_dense(const KInfo* kinfo, const double2* diag, const int64_t* offD,
                                 int n_k, double2* H, cudaStream_t s);
cudaError_t launch_mubar_reduce(const KInfo* kinfo, const SInfo* sinfo, int n_sys, int n_chunks,
                                const double* mubar_part, double* out, cudaStream_t s);

// Coefficient of M2 in rho_k: (2/beta) sum_{n<n_iw} 1/w_n^2 - beta/4 for tail_order 2
// (= -(beta / (2 pi^2)) psi'(n_iw + 1/2)), 0 for tail_order 1.
double tail_coefficient(double beta, int n_iw, int tail_order);

// Message returned by gf_last_error(NULL) (calls that have no context).  Never throws: if the
// message cannot be stored the previous one is cleared.
void set_global_error(const char* msg) noexcept;

// Status of the C++ exception being handled (call only inside a catch block): GF_ENOMEM for a
// failed or oversized host allocation, GF_EINVAL for anything else; *msg describes it.
inline gf_status exception_status(const char** msg) noexcept {
  try {
    throw;
  } catch (const std::bad_alloc&) {
    *msg = "host allocation failed";
    return GF_ENOMEM;
  } catch (const std::length_error&) {
    *msg = "host allocation too large";
    return GF_ENOMEM;
  } catch (...) {
    *msg = "unexpected C++ exception in host code";
    return GF_EINVAL;
  }
}

// Handler of the function-try-block around an entry point that has no context: the status of
// the exception, with its message for gf_last_error(NULL).
inline gf_status caught_global() noexcept {
  const char* msg = "";
  const gf_status s = exception_status(&msg);
  set_global_error(msg);
  return s;
}

}  // namespace gf

// Internal declarations shared by the CUDA translation units of libgf.
// Nothing here is part of the C-ABI (include/gf.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gf {

constexpr int kThreads = 256;          // threads per CTA of every point kernel
constexpr int kFlagSingular = 1;       // status bit: zero or non-finite pivot

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

struct Item {           // one unit of work: k-point k, frequencies [n0, n1)
  int k, n0, n1, chunk;
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
  // outputs
  double* occ_part;     // [n_k][n_chunks][2]
  double2* rho_part;    // [n_chunks][sum_k N_b^2]
  int64_t rho_chunk_stride;
  double2* gq;          // [k - kb0][n][mmax^2]
  int kb0;
  int n_iw;
  // adjoint
  const double2* gbar;  // [sum_s n_iw m_s^2] or null
  const double* nbar;   // [n_sys] device, or null
  double* mubar_part;   // [n_k][n_chunks]
  int* status;
};

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

__host__ __device__ inline int imax(int a, int b) { return a > b ? a : b; }

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
cudaError_t launch_gq_reduce(const KInfo* kinfo, const SInfo* sinfo, int n_sys, int max_mm_total,
                             const double2* gq, int kb0, int kb1, int n_iw, int mmax, int first,
                             double2* acc, cudaStream_t s);
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

// Message returned by gf_last_error(NULL) (calls that have no context).
void set_global_error(const char* msg);

}  // namespace gf

// The DMFT self-consistency step around the lattice sums (sm_103a).
//
//   k_eimp_part, k_eimp_reduce E_imp = sum_k w_k P_k H_k P_k^+ - V_DC I   (Eq. E^imp)
//   k_hybridization            Delta(i w_n) = (i w_n + mu) I - E_imp - Sigma(i w_n)
//                                             - G_loc(i w_n)^{-1}          (Eq. dmftloop2)
//                              one warp per (system, frequency): m x m inverse
//                              by Gauss-Jordan on [G_loc | I] in shared memory
// (The orthonormal projectors of Eqs. 6 and 7, k_lowdin, live in gf_eig.cu
// beside the Jacobi eigensolver they use.)
#include <math.h>
#include <stdint.h>

#include "gf_complex.cuh"
#include "gf_internal.cuh"

namespace gf {

namespace {

using namespace cx;


// part[k][a][b] = w_k (P_k H_k P_k^+)_{ab}, one CTA per k: T = H P^+ (N x m)
// in shared memory, then P T.
__global__ void __launch_bounds__(kThreads)
    k_eimp_part(const KInfo* __restrict__ kinfo, const SInfo* __restrict__ sinfo,
                const double2* __restrict__ H, const double2* __restrict__ P, int mmax,
                double2* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smraw[];
  double2* T = reinterpret_cast<double2*>(smraw);
  const int k = blockIdx.x;
  const KInfo ki = kinfo[k];
  const int N = ki.nb, M = sinfo[ki.sys].m;
  const double2* Hk = H + ki.offH;
  const double2* Pk = P + ki.offP;
  for (int e = threadIdx.x; e < N * M; e += kThreads) {
    const int j = e / M, b = e - (e / M) * M;
    double2 acc = make_double2(0.0, 0.0);
    for (int i = 0; i < N; ++i) cmac_cb(acc, Hk[j * N + i], Pk[b * N + i]);
    T[e] = acc;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < M * M; e += kThreads) {
    const int a = e / M, b = e - (e / M) * M;
    double2 acc = make_double2(0.0, 0.0);
    for (int j = 0; j < N; ++j) cmac(acc, Pk[a * N + j], T[j * M + b]);
    part[(int64_t)k * mmax * mmax + e] = make_double2(ki.w * acc.x, ki.w * acc.y);
  }
}

// out[s][e] = sum over the k of system s, in increasing k, of part[k][e] (m_s^2 entries),
// minus v_dc[s] on the diagonal.
__global__ void k_eimp_reduce(const SInfo* __restrict__ sinfo, const double2* __restrict__ part,
                              int mmax, const double* __restrict__ v_dc, double2* __restrict__ out) {
  const SInfo si = sinfo[blockIdx.x];
  const int M = si.m;
  for (int e = threadIdx.x; e < M * M; e += blockDim.x) {
    double2 acc = make_double2(0.0, 0.0);
    for (int k = si.k0; k < si.k1; ++k) {
      const double2 v = part[(int64_t)k * mmax * mmax + e];
      acc.x += v.x;
      acc.y += v.y;
    }
    const int a = e / M, b = e - (e / M) * M;
    if (a == b && v_dc) acc.x -= v_dc[blockIdx.x];
    out[si.offSinf + e] = acc;
  }
}

constexpr int kHybWarps = 4;

// Delta for one (system, frequency) per warp; lane i owns row i of [G | I].
__global__ void __launch_bounds__(32 * kHybWarps)
    k_hybridization(const SInfo* __restrict__ sinfo, int n_sys, int n_iw, int mmax,
                    const double* __restrict__ mu, const double2* __restrict__ eimp,
                    const double2* __restrict__ Sig, const double2* __restrict__ gloc,
                    double2* __restrict__ delta, int* status) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int task = blockIdx.x * kHybWarps + warp;
  if (task >= n_sys * n_iw) return;
  const int s = task / n_iw, n = task - (task / n_iw) * n_iw;
  const SInfo si = sinfo[s];
  const int M = si.m, W = 2 * M;
  double2* aug = reinterpret_cast<double2*>(smraw) + (size_t)warp * mmax * 2 * mmax;
  const double2* G = gloc + si.offSig + (int64_t)n * M * M;
  for (int e = lane; e < M * W; e += 32) {
    const int i = e / W, c = e - (e / W) * W;
    aug[e] = c < M ? G[i * M + c] : make_double2(c - M == i ? 1.0 : 0.0, 0.0);
  }
  __syncwarp();
  bool singular = false;
  for (int j = 0; j < M; ++j) {
    unsigned long long best = 0ULL;
    int bi = 0x7fffffff;
    for (int i = j + lane; i < M; i += 32) {
      const unsigned long long key = pivot_key(aug[i * W + j]);
      if (bi == 0x7fffffff || key > best) { best = key; bi = i; }
    }
    for (int off = 16; off; off >>= 1) {
      const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, off);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (best == 0ULL || best >= 0x7ff0000000000000ULL) singular = true;
    if (bi != j)
      for (int c = lane; c < W; c += 32) {
        const double2 t = aug[j * W + c];
        aug[j * W + c] = aug[bi * W + c];
        aug[bi * W + c] = t;
      }
    __syncwarp();
    const double2 r = crcp(aug[j * W + j]);
    __syncwarp();
    for (int c = lane; c < W; c += 32) aug[j * W + c] = c == j ? make_double2(1.0, 0.0) : cmul(aug[j * W + c], r);
    __syncwarp();
    for (int i = lane; i < M; i += 32) {
      if (i == j) continue;
      const double2 l = aug[i * W + j];
      for (int c = 0; c < W; ++c) {
        const double2 u = aug[j * W + c];
        double2 v = aug[i * W + c];
        v.x = fma(-l.x, u.x, fma(l.y, u.y, v.x));
        v.y = fma(-l.x, u.y, fma(-l.y, u.x, v.y));
        aug[i * W + c] = v;
      }
      aug[i * W + j] = make_double2(0.0, 0.0);
    }
    __syncwarp();
  }
  if (singular && lane == 0) atomicOr(status, kFlagSingular);
  const double wn = (2.0 * n + 1.0) * 3.14159265358979323846 / si.beta;
  const double2* Sg = Sig + si.offSig + (int64_t)n * M * M;
  const double2* E = eimp + si.offSinf;
  double2* D = delta + si.offSig + (int64_t)n * M * M;
  for (int e = lane; e < M * M; e += 32) {
    const int i = e / M, c = e - (e / M) * M;
    const double2 g = aug[i * W + M + c], sg = Sg[e], ei = E[e];
    double2 v = make_double2(-ei.x - sg.x - g.x, -ei.y - sg.y - g.y);
    if (i == c) {
      v.x += mu[s];
      v.y += wn;
    }
    D[e] = v;
  }
}

}  // namespace

cudaError_t launch_eimp(const KInfo* kinfo, const SInfo* sinfo, int n_k, int n_sys, const double2* H,
                        const double2* P, int nbmax, int mmax, double2* part, const double* v_dc,
                        double2* out, cudaStream_t s) {
  const size_t smem = (size_t)nbmax * mmax * sizeof(double2);
  cudaError_t e0 = cudaFuncSetAttribute(k_eimp_part, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e0 != cudaSuccess) return e0;
  k_eimp_part<<<n_k, kThreads, smem, s>>>(kinfo, sinfo, H, P, mmax, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_eimp_reduce<<<n_sys, kThreads, 0, s>>>(sinfo, part, mmax, v_dc, out);
  return cudaGetLastError();
}

cudaError_t launch_hybridization(const SInfo* sinfo, int n_sys, int n_iw, int mmax, const double* mu,
                                 const double2* eimp, const double2* Sig, const double2* gloc,
                                 double2* delta, int* status, cudaStream_t s) {
  const size_t smem = (size_t)kHybWarps * mmax * 2 * mmax * sizeof(double2);
  cudaError_t e =
      cudaFuncSetAttribute(k_hybridization, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int tasks = n_sys * n_iw;
  const int grid = (tasks + kHybWarps - 1) / kHybWarps;
  k_hybridization<<<grid, 32 * kHybWarps, smem, s>>>(sinfo, n_sys, n_iw, mmax, mu, eimp, Sig, gloc,
                                                      delta, status);
  return cudaGetLastError();
}

}  // namespace gf

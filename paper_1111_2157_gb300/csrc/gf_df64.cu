// FP32-pair ("df64") kernel of the lattice Green's function path (sm_103a).
//
// GB300 executes FP64 at 1/62 of the FP32 rate (about 2 DFMA per clock per SM
// against 128 FFMA).  An FP64 iterative-refinement residual I - A X costs N_b^3
// FP64 multiply-adds, as much as the FP64 inverse itself, so refinement in FP64
// cannot make a faster path on this chip.  This kernel instead carries every
// matrix entry as an unevaluated sum hi + lo of two FP32 numbers and does the
// embedding and the Gauss-Jordan inverse with error-free transformations on the
// FP32 pipes:
//   two_sum     (Knuth)   s + e = a + b exactly,        6 FP32 operations
//   two_prod    (FMA)     p + e = a * b exactly,        2 FP32 operations
// which gives about 2^-48 relative precision per operation (FP64 has 2^-53)
// at about 60 FP32 instructions per complex multiply-add.  The reductions that
// feed N(mu), rho_k and G_loc are accumulated in FP64, as is everything after
// the point kernel (the Matsubara tail, the k-sums and the mu search).
//
// Work items, modes, shared-memory layout and outputs are those of the FP64
// kernel (gf_fp64.cu); only the arithmetic of a1, a2 and the epilogue
// products differs.  gf_df64r.cu holds the register-resident variant; the
// library times both on first use and keeps the faster (gf_api.cu).  Complex pairs are stored as float4 {re.hi, re.lo, im.hi, im.lo}.
#include <math.h>
#include <stdint.h>

#include "gf_complex.cuh"
#include "gf_internal.cuh"

namespace gf {

namespace {

using namespace cx;

// ---------------------------------------------------------------- FP32 pairs
// The _rn intrinsics keep nvcc from contracting a product into a later add or
// reassociating the sums, which would break the error-free transformations.









__device__ __forceinline__ double block_sum_d(double v, double* red) {
  for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double r = 0.0;
  if (warp == 0) {
    r = lane < (kThreads / 32) ? red[lane] : 0.0;
    for (int off = 16; off; off >>= 1) r += __shfl_xor_sync(0xffffffffu, r, off);
  }
  return r;
}

// Pivot search of column j over rows j..N-1 by one warp; lane 0 stores the
// pivot row and the pair reciprocal of the pivot.
__device__ __forceinline__ void pivot_warp(const float4* A, int N, int ld, int j, int lane, int* s_p,
                                           float4* s_r, int* piv, int* status) {
  unsigned best = 0u;
  int bi = 0x7fffffff;
  for (int i = j + lane; i < N; i += 32) {
    const unsigned key = pivot_key_f(A[i * ld + j]);
    if (bi == 0x7fffffff || key > best) { best = key; bi = i; }
  }
  for (int off = 16; off; off >>= 1) {
    const unsigned ob = __shfl_xor_sync(0xffffffffu, best, off);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
    if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
  }
  if (lane == 0) {
    const cf pv = ld4(A[bi * ld + j]);
    if (best == 0u || best >= 0x7f800000u) atomicOr(status, kFlagSingular);
    *s_p = bi;
    *s_r = st4(crcp_df(pv));
    piv[j] = bi;
  }
}


__device__ __forceinline__ void elim_entry(float4* A, int ld, const float4* col, const float4* urow,
                                           int i, int c, int j) {
  float4* a = &A[i * ld + c];
  const float4 u4 = urow[c];
  if (i == j) {
    *a = u4;
  } else {
    const cf l = cneg(ld4(col[i]));
    const float4 a0 = *a;
    cf v = (c == j) ? czero() : ld4(a0);
    cacc(v, l, ld4(u4));
    renorm_fast(v.rh, v.rl);
    renorm_fast(v.ih, v.il);
    *a = st4(v);
  }
}

// In-place Gauss-Jordan inversion in FP32-pair arithmetic with one pivot of
// lookahead; the same pivoting and bookkeeping as the FP64 kernel (pivot key
// from the head words).  Step j: (b) scaled pivot row to urow, old row j to row
// p, column j to col; (c) warp 0 eliminates column j+1 first, then searches it
// for the next pivot and forms its reciprocal, while warps 1..7 eliminate every
// other column.  Two barriers per pivot; the pivot search is off the critical path.
__device__ void gauss_jordan_df64(float4* A, int N, int ld, float4* col, float4* urow, int* piv,
                                  int* idx, int* status) {
  __shared__ int s_p[2];
  __shared__ float4 s_r[2];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (warp == 0) pivot_warp(A, N, ld, 0, lane, &s_p[0], &s_r[0], piv, status);
  __syncthreads();
  for (int j = 0; j < N; ++j) {
    const int bf = j & 1;
    const int pr = s_p[bf];
    const cf r = ld4(s_r[bf]);
    for (int c = tid; c < N; c += kThreads) {
      const cf vp = ld4(A[pr * ld + c]);
      if (c == j) {
        urow[c] = st4(r);
      } else {
        cf u = czero();
        cacc(u, vp, r);
        cnorm(u);
        urow[c] = st4(u);
      }
      if (pr != j) A[pr * ld + c] = A[j * ld + c];
    }
    for (int i = tid; i < N; i += kThreads) col[i] = (i == pr) ? A[j * ld + j] : A[i * ld + j];
    __syncthreads();
    const int jn = j + 1;
    if (jn < N && warp == 0) {
      for (int i = lane; i < N; i += 32) elim_entry(A, ld, col, urow, i, jn, j);
      __syncwarp();
      pivot_warp(A, N, ld, jn, lane, &s_p[bf ^ 1], &s_r[bf ^ 1], piv, status);
    } else {
      // every (i, c) with c != jn, over warps 1..7 (all warps on the last step)
      const int w0 = (jn < N) ? 32 : 0;
      const int nt = kThreads - w0, me = tid - w0;
      const int ncol = (jn < N) ? N - 1 : N;
      const int total = N * ncol;
      int i = me / ncol, cc = me - (me / ncol) * ncol;
      const int di = nt / ncol, dc = nt - (nt / ncol) * ncol;
      for (int e = me; e < total; e += nt) {
        elim_entry(A, ld, col, urow, i, cc + (cc >= jn ? 1 : 0), j);
        i += di; cc += dc;
        if (cc >= ncol) { cc -= ncol; ++i; }
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    for (int c = 0; c < N; ++c) idx[c] = c;
    for (int j = N - 1; j >= 0; --j) {
      const int p = piv[j];
      if (p != j) { const int t = idx[j]; idx[j] = idx[p]; idx[p] = t; }
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kThreads) k_point_df64(const PointParams p) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float4* sm = reinterpret_cast<float4*>(smraw);
  __shared__ int s_item;
  __shared__ double s_red[kThreads / 32];
  const Layout L = make_layout(p.nbmax, p.mmax, p.mode, p.a_in_smem);
  float4* sP = sm + L.offP;
  float4* sT = sm + L.offT;
  float4* sZ = sm + L.offZ;
  float4* sS = sm + L.offS;
  float4* sQa = sm + L.offQa;
  float4* sQb = sm + L.offQb;
  float4* sCol = sm + L.offCol;
  float4* sU = sm + L.offU;
  int* sPiv = reinterpret_cast<int*>(sm + L.n2);
  int* sIdx = sPiv + p.nbmax;
  const int tid = threadIdx.x;

  for (;;) {
    if (tid == 0) s_item = atomicAdd(p.queue, 1);
    __syncthreads();
    const int itx = s_item;
    if (itx >= p.n_items) break;
    const Item it = p.items[itx];
    for (int q = 0; q < it.nk; ++q) {
      const int kk = item_k(it, p.kperm, q);
      const KInfo ki = p.kinfo[kk];
      const SInfo si = p.sinfo[ki.sys];
      const int N = ki.nb, M = si.m, ld = N | 1;
      float4* A = p.a_in_smem ? (sm + L.offA)
                              : reinterpret_cast<float4*>(p.a_scratch + (int64_t)blockIdx.x * p.a_stride);
      const float4* Hk = p.Hd + ki.offH;
      const float4* Pg = p.Pd + ki.offP;
      const double mu = p.mu[ki.sys];
      const double beta = si.beta;
      const double wk = ki.w;
      double nbar = 0.0;
      if ((p.mode & kAdj) && p.nbar) nbar = p.nbar[ki.sys];
      float mu_h, mu_l;
      split(mu, mu_h, mu_l);
      for (int e = tid; e < M * N; e += kThreads) sP[e] = Pg[e];

      double acc_tr = 0.0, acc_mu = 0.0;
      float g2h = 0.f, g2l = 0.f;
      for (int n = it.n0; n < it.n1; ++n) {
        const double wn = (2.0 * n + 1.0) * M_PI / beta;
        float wn_h, wn_l;
        split(wn, wn_h, wn_l);
        const float4* Sg = p.Sd + si.offSig + (int64_t)n * M * M;
        __syncthreads();
        for (int e = tid; e < M * M; e += kThreads) sS[e] = Sg[e];
        __syncthreads();
        // T = Sigma(i w_n) P_k
        for (int e = tid; e < M * N; e += kThreads) {
          const int a = e / N, j = e - a * N;
          cf acc = czero();
          for (int b = 0; b < M; ++b) cacc(acc, ld4(sS[a * M + b]), ld4(sP[b * N + j]));
          cnorm(acc);
          sT[e] = st4(acc);
        }
        __syncthreads();
        // A = (i w_n + mu) I - H_k - P_k^+ T
        for (int e = tid; e < N * N; e += kThreads) {
          const int i = e / N, j = e - i * N;
          cf acc = cneg(ld4(Hk[e]));
          if (i == j) {
            float s, t;
            two_sum(acc.rh, mu_h, s, t);
            acc.rh = s;
            acc.rl = __fadd_rn(acc.rl, __fadd_rn(t, mu_l));
            two_sum(acc.ih, wn_h, s, t);
            acc.ih = s;
            acc.il = __fadd_rn(acc.il, __fadd_rn(t, wn_l));
          }
          for (int a = 0; a < M; ++a) cacc_ca(acc, cneg(ld4(sP[a * N + i])), ld4(sT[a * N + j]));
          cnorm(acc);
          A[i * ld + j] = st4(acc);
        }
        __syncthreads();
        gauss_jordan_df64(A, N, ld, sCol, sU, sPiv, sIdx, p.status);

        if (p.mode & kOcc) {
          for (int i = tid; i < N; i += kThreads) {
            const float4 g = A[i * ld + sIdx[i]];
            acc_tr += (double)g.x + (double)g.y;
          }
          for (int e = tid; e < N * N; e += kThreads) {
            const int i = e / N, c = e - i * N;
            const float4 g1 = A[i * ld + sIdx[c]], g2 = A[c * ld + sIdx[i]];
            acc_prod(g1.x, g1.y, g2.x, g2.y, g2h, g2l);
            acc_prod(-g1.z, -g1.w, g2.z, g2.w, g2h, g2l);
          }
          renorm(g2h, g2l);
        }
        if (p.mode & kRho) {
          double2* S = p.rho_part + (int64_t)it.chunk * p.rho_chunk_stride + ki.offH;
          const bool first = (n == it.n0);
          for (int e = tid; e < N * N; e += kThreads) {
            const int i = e / N, c = e - i * N;
            const double2 g = to_d2(ld4(A[i * ld + sIdx[c]]));
            if (first) {
              S[e] = g;
            } else {
              double2 s = S[e];
              s.x += g.x;
              s.y += g.y;
              S[e] = s;
            }
          }
        }
        if (p.mode & (kGloc | kAdj)) {
          for (int e = tid; e < N * M; e += kThreads) {
            const int i = e / M, b = e - i * M;
            cf acc = czero();
            for (int c = 0; c < N; ++c) {
              cacc_cb(acc, ld4(A[i * ld + sIdx[c]]), ld4(sP[b * N + c]));
              if ((c & 15) == 15) cnorm(acc);
            }
            cnorm(acc);
            sT[e] = st4(acc);
          }
          if (p.mode & kAdj) {
            for (int e = tid; e < M * N; e += kThreads) {
              const int a = e / N, c = e - a * N;
              const int colx = sIdx[c];
              cf acc = czero();
              for (int i = 0; i < N; ++i) {
                cacc(acc, ld4(sP[a * N + i]), ld4(A[i * ld + colx]));
                if ((i & 15) == 15) cnorm(acc);
              }
              cnorm(acc);
              sZ[e] = st4(acc);
            }
          }
          __syncthreads();
        }
        if (p.mode & kGloc) {
          double2* out = p.gq + ((int64_t)(it.g - p.gb0) * p.n_iw + n) * p.mmax * p.mmax;
          for (int e = tid; e < M * M; e += kThreads) {
            const int a = e / M, b = e - a * M;
            cf acc = czero();
            for (int i = 0; i < N; ++i) {
              cacc(acc, ld4(sP[a * N + i]), ld4(sT[i * M + b]));
              if ((i & 15) == 15) cnorm(acc);
            }
            cnorm(acc);
            const double2 qv = to_d2(acc);
            gq_put(&out[e], q, make_double2(wk * qv.x, wk * qv.y));
          }
        }
        if (p.mode & kAdj) {
          for (int e = tid; e < M * M; e += kThreads) {
            const int a = e / M, b = e - a * M;
            cf aa = czero(), bb = czero();
            for (int i = 0; i < N; ++i) {
              const cf y = ld4(sT[i * M + b]);
              cacc(aa, ld4(sP[a * N + i]), y);
              cacc(bb, ld4(sZ[a * N + i]), y);
              if ((i & 15) == 15) { cnorm(aa); cnorm(bb); }
            }
            cnorm(aa);
            cnorm(bb);
            sQa[e] = st4(aa);
            sQb[e] = st4(bb);
          }
          __syncthreads();
          const bool have_gbar = (p.Gbd != nullptr);
          if (have_gbar) {
            const float4* Gb = p.Gbd + si.offSig + (int64_t)n * M * M;
            for (int e = tid; e < M * M; e += kThreads) sS[e] = Gb[e];
            __syncthreads();
            for (int e = tid; e < M * M; e += kThreads) {
              const int a = e / M, b = e - a * M;
              cf acc = czero();
              for (int c = 0; c < M; ++c) cacc_cb(acc, ld4(sS[a * M + c]), ld4(sQa[b * M + c]));
              cnorm(acc);
              sT[e] = st4(acc);
            }
            __syncthreads();
            for (int e = tid; e < M * M; e += kThreads) {
              const double2 g = to_d2(ld4(sS[e])), b = to_d2(ld4(sQb[e]));
              acc_mu -= wk * fma(g.x, b.x, g.y * b.y);
            }
          }
          double2* out = p.gq + ((int64_t)(it.g - p.gb0) * p.n_iw + n) * p.mmax * p.mmax;
          const double cb = nbar * 2.0 / beta;
          for (int e = tid; e < M * M; e += kThreads) {
            const int a = e / M, b = e - a * M;
            cf acc = czero();
            if (have_gbar)
              for (int c = 0; c < M; ++c) cacc_ca(acc, ld4(sQa[c * M + a]), ld4(sT[c * M + b]));
            cnorm(acc);
            const double2 v = to_d2(acc);
            const double2 bt = to_d2(ld4(sQb[b * M + a]));
            gq_put(&out[e], q, make_double2(wk * fma(cb, bt.x, v.x), wk * fma(-cb, bt.y, v.y)));
          }
        }
      }
      if (p.mode & kOcc) {
        const double tr = block_sum_d(acc_tr, s_red);
        const double g2 = block_sum_d((double)g2h + (double)g2l, s_red);
        if (tid == 0) {
          double* o = p.occ_part + ((int64_t)kk * p.n_chunks + it.chunk) * 2;
          o[0] = tr;
          o[1] = g2;
        }
      }
      if (p.mode & kAdj) {
        const double mb = block_sum_d(acc_mu, s_red);
        if (tid == 0) p.mubar_part[(int64_t)kk * p.n_chunks + it.chunk] = mb;
      }
      __syncthreads();
    }
  }
}

__global__ void k_split_df64(const double2* __restrict__ in, float4* __restrict__ out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double2 v = in[i];
  float4 r;
  split(v.x, r.x, r.y);
  split(v.y, r.z, r.w);
  out[i] = r;
}

}  // namespace

cudaError_t launch_point_df64(const PointParams& p, int grid, size_t smem, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(k_point_df64, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_point_df64<<<grid, kThreads, smem, s>>>(p);
  return cudaGetLastError();
}

size_t point_df64_smem(int nbmax, int mmax, int mode, int a_in_smem, int /*nmat*/) {
  return make_layout(nbmax, mmax, mode, a_in_smem).bytes;
}

int point_df64_blocks_per_sm(size_t smem) {
  int nb = 0;
  cudaFuncSetAttribute(k_point_df64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_point_df64, kThreads, smem) != cudaSuccess)
    return 0;
  return nb;
}

cudaError_t launch_split_df64(const double2* in, float4* out, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_split_df64<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, out, n);
  return cudaGetLastError();
}

}  // namespace gf

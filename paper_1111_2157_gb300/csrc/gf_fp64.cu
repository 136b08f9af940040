// FP64 kernels of the lattice Green's function path (sm_103a).
//
// k_point_fp64 is a persistent kernel: each CTA takes work items (k, [n0, n1))
// from an atomic counter and, for every frequency of the item,
//   1. embeds   A = (i w_n + mu) I - H_k - P_k^+ (Sigma(i w_n) P_k)      (Eq. dmftloop1)
//   2. inverts  A in place by Gauss-Jordan elimination with partial pivoting
//   3. consumes G = A^{-1} in the epilogue selected by the mode bits:
//      kOcc  Re Tr G and Re Tr G^2          -> N(mu), dN/dmu  (Eq. fix_mu)
//      kRho  S_k += G                       -> rho_k          (Eq. rho_LDA+DMFT)
//      kGloc w_k P_k G P_k^+                -> G_loc          (Eq. dmftloop2)
//      kAdj  w_k [A^+ Gbar A^+ + nbar (2/beta) B^+], A = P G P^+, B = P G^2 P^+
// G(k, i w_n) itself never leaves the chip.  On GB300 the FP64 pipe (about
// 2 DFMA per clock per SM) is the bound, so the kernel keeps the matrix in
// shared memory, spends no FP64 instruction on pivot search (the pivot key is
// the integer bit pattern of max(|Re|, |Im|)) and lets every other unit run
// in the shadow of the DFMA stream.
#include <math.h>
#include <stdint.h>

#include "gf_complex.cuh"
#include "gf_internal.cuh"

namespace gf {

namespace {

using namespace cx;




__device__ __forceinline__ double block_sum(double v, double* red) {
  // Deterministic: fixed xor tree inside each warp, then warp 0 over the warps.
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
  return r;  // valid in thread 0
}

// In-place Gauss-Jordan inversion of the N x N matrix A (leading dimension ld)
// with partial pivoting.  On return A holds A^{-1} with its columns permuted:
// column c of the inverse is column idx[c] of A.  Three barriers per pivot.
__device__ void gauss_jordan_fp64(double2* A, int N, int ld, double2* col, double2* urow, int* piv,
                                  int* idx, int* status) {
  __shared__ int s_p;
  __shared__ double2 s_r;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int j = 0; j < N; ++j) {
    if (warp == 0) {
      unsigned long long best = 0ULL;
      int bi = 0x7fffffff;
      for (int i = j + lane; i < N; i += 32) {
        const unsigned long long key = pivot_key(A[i * ld + j]);
        if (bi == 0x7fffffff || key > best) { best = key; bi = i; }
      }
      for (int off = 16; off; off >>= 1) {
        const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, off);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (lane == 0) {
        const double2 pv = A[bi * ld + j];
        if (best == 0ULL || best >= 0x7ff0000000000000ULL) atomicOr(status, kFlagSingular);
        s_p = bi;
        s_r = crcp(pv);
        piv[j] = bi;
      }
    }
    __syncthreads();
    const int pr = s_p;
    const double2 r = s_r;
    // Scaled pivot row into urow, old row j moved to row pr, column j saved in
    // the post-swap row order.  Only row pr is written: no other thread reads it.
    for (int c = tid; c < N; c += kThreads) {
      const double2 vp = A[pr * ld + c];
      urow[c] = (c == j) ? r : cmul(vp, r);
      if (pr != j) A[pr * ld + c] = A[j * ld + c];
    }
    for (int i = tid; i < N; i += kThreads) col[i] = (i == pr) ? A[j * ld + j] : A[i * ld + j];
    __syncthreads();
    // Eliminate column j from every other row; column j receives the inverse's
    // entries.  One branch-free update a' = a - l u for every element: row j takes
    // l = 0, a = urow (so a' = urow), column j takes a = 0 (so a' = -l r, since
    // urow[j] = r).  The selects keep divergent FP64 paths out of the warps.
    const int total = N * N;
    int i = tid / N, c = tid - (tid / N) * N;
    const int di = kThreads / N, dc = kThreads - (kThreads / N) * N;
    const double2 zero = make_double2(0.0, 0.0);
    for (int e = tid; e < total; e += kThreads) {
      double2* a = &A[i * ld + c];
      const double2 u = urow[c];
      const double2 l = (i == j) ? zero : col[i];
      const double2 a0 = *a;
      double2 v = (i == j) ? u : ((c == j) ? zero : a0);
      v.x = fma(-l.x, u.x, fma(l.y, u.y, v.x));
      v.y = fma(-l.x, u.y, fma(-l.y, u.x, v.y));
      *a = v;
      i += di; c += dc;
      if (c >= N) { c -= N; ++i; }
    }
    __syncthreads();
  }
  // Undoing the row interchanges permutes columns in reverse order; record the
  // composed permutation instead of moving data.
  if (tid == 0) {
    for (int c = 0; c < N; ++c) idx[c] = c;
    for (int j = N - 1; j >= 0; --j) {
      const int p = piv[j];
      if (p != j) { const int t = idx[j]; idx[j] = idx[p]; idx[p] = t; }
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kThreads) k_point_fp64(const PointParams p) {
  extern __shared__ __align__(16) unsigned char smraw[];
  double2* sm = reinterpret_cast<double2*>(smraw);
  __shared__ int s_item;
  __shared__ double s_red[kThreads / 32];
  const Layout L = make_layout(p.nbmax, p.mmax, p.mode, p.a_in_smem);
  double2* sP = sm + L.offP;
  double2* sT = sm + L.offT;
  double2* sZ = sm + L.offZ;
  double2* sS = sm + L.offS;
  double2* sQa = sm + L.offQa;
  double2* sQb = sm + L.offQb;
  double2* sCol = sm + L.offCol;
  double2* sU = sm + L.offU;
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
      double2* A = p.a_in_smem ? (sm + L.offA) : (p.a_scratch + (int64_t)blockIdx.x * p.a_stride);
      const double2* Hk = p.H + ki.offH;
      const double2* Pg = p.P + ki.offP;
      const double mu = p.mu[ki.sys];
      const double beta = si.beta;
      const double wk = ki.w;
      double nbar = 0.0;
      if ((p.mode & kAdj) && p.nbar) nbar = p.nbar[ki.sys];
      for (int e = tid; e < M * N; e += kThreads) sP[e] = Pg[e];

      double acc_tr = 0.0, acc_g2 = 0.0, acc_mu = 0.0;
      for (int n = it.n0; n < it.n1; ++n) {
        const double wn = (2.0 * n + 1.0) * M_PI / beta;
        const double2* Sg = p.Sig + si.offSig + (int64_t)n * M * M;
        __syncthreads();  // previous epilogue done with sS / sT; sP loaded
        for (int e = tid; e < M * M; e += kThreads) sS[e] = Sg[e];
        __syncthreads();
        // T = Sigma(i w_n) P_k   (M x N)
        for (int e = tid; e < M * N; e += kThreads) {
          const int a = e / N, j = e - a * N;
          double2 acc = make_double2(0.0, 0.0);
          for (int b = 0; b < M; ++b) cmac(acc, sS[a * M + b], sP[b * N + j]);
          sT[e] = acc;
        }
        __syncthreads();
        // A = (i w_n + mu) I - H_k - P_k^+ T, accumulated as d - H - sum_a conj(P_ai) T_aj
        for (int e = tid; e < N * N; e += kThreads) {
          const int i = e / N, j = e - i * N;
          const double2 h = Hk[e];
          double2 v = make_double2((i == j ? mu : 0.0) - h.x, (i == j ? wn : 0.0) - h.y);
          for (int a = 0; a < M; ++a) {
            const double2 p = sP[a * N + i], t = sT[a * N + j];
            v.x = fma(-p.x, t.x, fma(-p.y, t.y, v.x));
            v.y = fma(-p.x, t.y, fma(p.y, t.x, v.y));
          }
          A[i * ld + j] = v;
        }
        __syncthreads();
        gauss_jordan_fp64(A, N, ld, sCol, sU, sPiv, sIdx, p.status);
        // G[i][c] = A[i * ld + sIdx[c]]

        if (p.mode & kOcc) {
          for (int i = tid; i < N; i += kThreads) acc_tr += A[i * ld + sIdx[i]].x;
          for (int e = tid; e < N * N; e += kThreads) {
            const int i = e / N, c = e - i * N;
            const double2 g1 = A[i * ld + sIdx[c]], g2 = A[c * ld + sIdx[i]];
            acc_g2 = fma(g1.x, g2.x, fma(-g1.y, g2.y, acc_g2));
          }
        }
        if (p.mode & kRho) {
          double2* S = p.rho_part + (int64_t)it.chunk * p.rho_chunk_stride + ki.offH;
          const bool first = (n == it.n0);
          for (int e = tid; e < N * N; e += kThreads) {
            const int i = e / N, c = e - i * N;
            const double2 g = A[i * ld + sIdx[c]];
            if (first) {
              S[e] = g;
            } else {
              double2 s = S[e];
              s.x += g.x; s.y += g.y;
              S[e] = s;
            }
          }
        }
        if (p.mode & (kGloc | kAdj)) {
          // Y = G P^+ (N x M), in sT
          for (int e = tid; e < N * M; e += kThreads) {
            const int i = e / M, b = e - i * M;
            double2 acc = make_double2(0.0, 0.0);
            for (int c = 0; c < N; ++c) cmac_cb(acc, A[i * ld + sIdx[c]], sP[b * N + c]);
            sT[e] = acc;
          }
          if (p.mode & kAdj) {
            // Z = P G (M x N)
            for (int e = tid; e < M * N; e += kThreads) {
              const int a = e / N, c = e - a * N;
              double2 acc = make_double2(0.0, 0.0);
              const int col = sIdx[c];
              for (int i = 0; i < N; ++i) cmac(acc, sP[a * N + i], A[i * ld + col]);
              sZ[e] = acc;
            }
          }
          __syncthreads();
        }
        if (p.mode & kGloc) {
          double2* out = p.gq + ((int64_t)(it.g - p.gb0) * p.n_iw + n) * p.mmax * p.mmax;
          for (int e = tid; e < M * M; e += kThreads) {
            const int a = e / M, b = e - a * M;
            double2 acc = make_double2(0.0, 0.0);
            for (int i = 0; i < N; ++i) cmac(acc, sP[a * N + i], sT[i * M + b]);
            gq_put(&out[e], q, make_double2(wk * acc.x, wk * acc.y));
          }
        }
        if (p.mode & kAdj) {
          // A_k = P Y, B_k = Z Y  (M x M)
          for (int e = tid; e < M * M; e += kThreads) {
            const int a = e / M, b = e - a * M;
            double2 aa = make_double2(0.0, 0.0), bb = make_double2(0.0, 0.0);
            for (int i = 0; i < N; ++i) {
              const double2 y = sT[i * M + b];
              cmac(aa, sP[a * N + i], y);
              cmac(bb, sZ[a * N + i], y);
            }
            sQa[e] = aa;
            sQb[e] = bb;
          }
          __syncthreads();
          const bool have_gbar = (p.gbar != nullptr);
          if (have_gbar) {
            const double2* Gb = p.gbar + si.offSig + (int64_t)n * M * M;
            for (int e = tid; e < M * M; e += kThreads) sS[e] = Gb[e];
            __syncthreads();
            // Mt = Gbar A^+  (M x M), in sT
            for (int e = tid; e < M * M; e += kThreads) {
              const int a = e / M, b = e - a * M;
              double2 acc = make_double2(0.0, 0.0);
              for (int c = 0; c < M; ++c) cmac_cb(acc, sS[a * M + c], sQa[b * M + c]);
              sT[e] = acc;
            }
            __syncthreads();
            // mu_bar partial: - w_k Re<Gbar, B>
            for (int e = tid; e < M * M; e += kThreads) {
              const double2 g = sS[e], b = sQb[e];
              acc_mu -= wk * fma(g.x, b.x, g.y * b.y);
            }
          }
          double2* out = p.gq + ((int64_t)(it.g - p.gb0) * p.n_iw + n) * p.mmax * p.mmax;
          const double cb = nbar * 2.0 / beta;
          for (int e = tid; e < M * M; e += kThreads) {
            const int a = e / M, b = e - a * M;
            double2 acc = make_double2(0.0, 0.0);
            if (have_gbar)
              for (int c = 0; c < M; ++c) cmac_ca(acc, sQa[c * M + a], sT[c * M + b]);
            const double2 bt = sQb[b * M + a];  // (B^+)_{ab} = conj(B_{ba})
            acc.x = fma(cb, bt.x, acc.x);
            acc.y = fma(-cb, bt.y, acc.y);
            gq_put(&out[e], q, make_double2(wk * acc.x, wk * acc.y));
          }
        }
      }
      // Item end: deterministic block reductions of the per-thread partials.
      if (p.mode & kOcc) {
        const double tr = block_sum(acc_tr, s_red);
        const double g2 = block_sum(acc_g2, s_red);
        if (tid == 0) {
          double* o = p.occ_part + ((int64_t)kk * p.n_chunks + it.chunk) * 2;
          o[0] = tr;
          o[1] = g2;
        }
      }
      if (p.mode & kAdj) {
        const double mb = block_sum(acc_mu, s_red);
        if (tid == 0) p.mubar_part[(int64_t)kk * p.n_chunks + it.chunk] = mb;
      }
      __syncthreads();
    }
  }
}

// N_k = (2/beta) Re Tr S_k + tailc Tr M2_k + N_b/2 and
// dN_k/dmu = -(2/beta) Re Tr sum_n G^2 - N_b tailc, with Tr M2_k = trHE_k - mu N_b.
__global__ void k_occ_finalize(const KInfo* __restrict__ kinfo, const SInfo* __restrict__ sinfo,
                               const double* __restrict__ trHE, const double* __restrict__ mu,
                               const double* __restrict__ occ_part, int n_chunks, int n_k,
                               double* __restrict__ kN, double* __restrict__ kdN) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_k) return;
  const KInfo ki = kinfo[k];
  const SInfo si = sinfo[ki.sys];
  double tr = 0.0, g2 = 0.0;
  for (int c = 0; c < n_chunks; ++c) {
    tr += occ_part[((int64_t)k * n_chunks + c) * 2 + 0];
    g2 += occ_part[((int64_t)k * n_chunks + c) * 2 + 1];
  }
  const double trM2 = trHE[k] - mu[ki.sys] * ki.nb;
  kN[k] = 2.0 / si.beta * tr + si.tailc * trM2 + 0.5 * ki.nb;
  kdN[k] = -2.0 / si.beta * g2 - ki.nb * si.tailc;
}

// out[s*2 + {0,1}] = sum_{k in s} w_k a[k], sum_{k in s} w_k b[k] (b may be null).
__global__ void __launch_bounds__(kThreads) k_sys_reduce(const KInfo* __restrict__ kinfo,
                                                         const SInfo* __restrict__ sinfo,
                                                         const double* __restrict__ a,
                                                         const double* __restrict__ b,
                                                         double* __restrict__ out) {
  __shared__ double red[kThreads / 32];
  const SInfo si = sinfo[blockIdx.x];
  double sa = 0.0, sb = 0.0;
  for (int k = si.k0 + threadIdx.x; k < si.k1; k += kThreads) {
    const double w = kinfo[k].w;
    sa = fma(w, a[k], sa);
    if (b) sb = fma(w, b[k], sb);
  }
  const double ra = block_sum(sa, red);
  const double rb = block_sum(sb, red);
  if (threadIdx.x == 0) {
    out[blockIdx.x * 2 + 0] = ra;
    out[blockIdx.x * 2 + 1] = rb;
  }
}

// rho_k = (S + S^+)/beta + tailc M2 + I/2, with S = sum of the chunk partials and
// M2 = H + E_inf - mu I.  One CTA per k; also N_k = Tr rho_k and
// n_corr,k = Tr(P rho P^+) = sum_ij rho_ij (P^+ P)_ji.
__global__ void __launch_bounds__(kThreads) k_rho_finalize(
    const KInfo* __restrict__ kinfo, const SInfo* __restrict__ sinfo, const double2* __restrict__ H,
    const double2* __restrict__ Einf, const double2* __restrict__ P, const double* __restrict__ mu,
    const double2* __restrict__ rho_part, int64_t stride, int n_chunks, double2* __restrict__ rho_out,
    double* __restrict__ kN, double* __restrict__ kNc) {
  __shared__ double red[kThreads / 32];
  const int k = blockIdx.x;
  const KInfo ki = kinfo[k];
  const SInfo si = sinfo[ki.sys];
  const int N = ki.nb, M = si.m;
  const double m0 = mu[ki.sys];
  const double2* Pk = P + ki.offP;
  double tr = 0.0, trc = 0.0;
  for (int e = threadIdx.x; e < N * N; e += kThreads) {
    const int i = e / N, j = e - i * N;
    double2 s = make_double2(0.0, 0.0), st = make_double2(0.0, 0.0);
    for (int c = 0; c < n_chunks; ++c) {
      const double2 a = rho_part[c * stride + ki.offH + e];
      const double2 b = rho_part[c * stride + ki.offH + j * N + i];
      s.x += a.x; s.y += a.y;
      st.x += b.x; st.y += b.y;
    }
    const double2 h = H[ki.offH + e], ei = Einf[ki.offH + e];
    double2 r;
    r.x = (s.x + st.x) / si.beta + si.tailc * (h.x + ei.x - (i == j ? m0 : 0.0));
    r.y = (s.y - st.y) / si.beta + si.tailc * (h.y + ei.y);
    if (i == j) r.x += 0.5;
    if (rho_out) rho_out[ki.offH + e] = r;
    if (i == j) tr += r.x;
    // (P^+ P)_ji = sum_a conj(P_aj) P_ai
    double2 pp = make_double2(0.0, 0.0);
    for (int a = 0; a < M; ++a) cmac_ca(pp, Pk[a * N + j], Pk[a * N + i]);
    trc = fma(r.x, pp.x, fma(-r.y, pp.y, trc));
  }
  const double t1 = block_sum(tr, red);
  const double t2 = block_sum(trc, red);
  if (threadIdx.x == 0) {
    kN[k] = t1;
    kNc[k] = t2;
  }
}

// acc[s][n][e] (+)= sum over the k-groups g of system s in [gb0, gb1) of gq[g - gb0][n][e], in
// increasing g (each group's slot already holds its k-points' sum in k order).
__global__ void k_gq_reduce(const SInfo* __restrict__ sinfo, const int* __restrict__ sys_g0,
                            const int* __restrict__ sys_g1, const double2* __restrict__ gq, int gb0,
                            int gb1, int n_iw, int mmax, int first, double2* __restrict__ acc) {
  const int s = blockIdx.y;
  const SInfo si = sinfo[s];
  const int M = si.m;
  const int64_t total = (int64_t)n_iw * M * M;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  const int n = (int)(t / (M * M));
  const int e = (int)(t - (int64_t)n * M * M);
  const int ga = sys_g0[s] > gb0 ? sys_g0[s] : gb0;
  const int gz = sys_g1[s] < gb1 ? sys_g1[s] : gb1;
  double2 v = first ? make_double2(0.0, 0.0) : acc[si.offSig + t];
  for (int g = ga; g < gz; ++g) {
    const double2 x = gq[((int64_t)(g - gb0) * n_iw + n) * mmax * mmax + e];
    v.x += x.x;
    v.y += x.y;
  }
  acc[si.offSig + t] = v;
}

// E_inf,k = P_k^+ Sigma_inf P_k and trHE_k = Re Tr(H_k + E_inf,k) (by trhe_partial).  One CTA
// per k.
__global__ void __launch_bounds__(kThreads) k_einf(const KInfo* __restrict__ kinfo,
                                                   const SInfo* __restrict__ sinfo,
                                                   const double2* __restrict__ H,
                                                   const double2* __restrict__ P,
                                                   const double2* __restrict__ Sinf,
                                                   double2* __restrict__ Einf,
                                                   double* __restrict__ trHE) {
  __shared__ double red[kThreads / 32];
  const int k = blockIdx.x;
  const KInfo ki = kinfo[k];
  const SInfo si = sinfo[ki.sys];
  const int N = ki.nb, M = si.m;
  const double2* Pk = P + ki.offP;
  const double2* S = Sinf + si.offSinf;
  for (int e = threadIdx.x; e < N * N; e += kThreads) {
    const int i = e / N, j = e - i * N;
    double2 v = make_double2(0.0, 0.0);
    for (int a = 0; a < M; ++a) {
      double2 t = make_double2(0.0, 0.0);
      for (int b = 0; b < M; ++b) cmac(t, S[a * M + b], Pk[b * N + j]);
      cmac_ca(v, Pk[a * N + i], t);
    }
    Einf[ki.offH + e] = v;
  }
  const double t = block_sum(trhe_partial(H + ki.offH, Pk, S, N, M, threadIdx.x, kThreads), red);
  if (threadIdx.x == 0) trHE[k] = t;
}

__global__ void k_upcast(const float2* __restrict__ in, double2* __restrict__ out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = make_double2((double)in[i].x, (double)in[i].y);
}

__global__ void k_diag_to_dense(const KInfo* __restrict__ kinfo, const double2* __restrict__ diag,
                                const int64_t* __restrict__ offD, double2* __restrict__ H) {
  const int k = blockIdx.x;
  const KInfo ki = kinfo[k];
  const int N = ki.nb;
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
    const int i = e / N, j = e - i * N;
    H[ki.offH + e] = (i == j) ? diag[offD[k] + i] : make_double2(0.0, 0.0);
  }
}

// out[s] = sum_{k in s} sum_c mubar_part[k][c] (fixed order).
__global__ void __launch_bounds__(kThreads) k_mubar_reduce(const SInfo* __restrict__ sinfo,
                                                           int n_chunks,
                                                           const double* __restrict__ part,
                                                           double* __restrict__ out) {
  __shared__ double red[kThreads / 32];
  const SInfo si = sinfo[blockIdx.x];
  double v = 0.0;
  for (int k = si.k0 + threadIdx.x; k < si.k1; k += kThreads)
    for (int c = 0; c < n_chunks; ++c) v += part[(int64_t)k * n_chunks + c];
  const double r = block_sum(v, red);
  if (threadIdx.x == 0) out[blockIdx.x] = r;
}

}  // namespace

size_t point_fp64_smem(int nbmax, int mmax, int mode, int a_in_smem) {
  return make_layout(nbmax, mmax, mode, a_in_smem).bytes;
}

cudaError_t launch_point_fp64(const PointParams& p, int grid, size_t smem, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(k_point_fp64, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_point_fp64<<<grid, kThreads, smem, s>>>(p);
  return cudaGetLastError();
}

int point_fp64_blocks_per_sm(size_t smem) {
  int nb = 0;
  cudaFuncSetAttribute(k_point_fp64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_point_fp64, kThreads, smem) != cudaSuccess)
    return 0;
  return nb;
}

cudaError_t launch_occ_finalize(const KInfo* kinfo, const SInfo* sinfo, const double* trHE,
                                const double* mu, const double* occ_part, int n_chunks, int n_k,
                                double* kN, double* kdN, cudaStream_t s) {
  k_occ_finalize<<<(n_k + 127) / 128, 128, 0, s>>>(kinfo, sinfo, trHE, mu, occ_part, n_chunks, n_k,
                                                   kN, kdN);
  return cudaGetLastError();
}

cudaError_t launch_sys_reduce(const KInfo* kinfo, const SInfo* sinfo, int n_sys, const double* a,
                              const double* b, double* out, cudaStream_t s) {
  k_sys_reduce<<<n_sys, kThreads, 0, s>>>(kinfo, sinfo, a, b, out);
  return cudaGetLastError();
}

cudaError_t launch_rho_finalize(const KInfo* kinfo, const SInfo* sinfo, const double2* H,
                                const double2* Einf, const double2* P, const double* mu,
                                const double2* rho_part, int64_t stride, int n_chunks, int n_k,
                                double2* rho_out, double* kN, double* kNc, cudaStream_t s) {
  k_rho_finalize<<<n_k, kThreads, 0, s>>>(kinfo, sinfo, H, Einf, P, mu, rho_part, stride, n_chunks,
                                          rho_out, kN, kNc);
  return cudaGetLastError();
}

cudaError_t launch_gq_reduce(const SInfo* sinfo, int n_sys, int max_mm_total, const int* sys_g0,
                             const int* sys_g1, const double2* gq, int gb0, int gb1, int n_iw,
                             int mmax, int first, double2* acc, cudaStream_t s) {
  dim3 grid((max_mm_total + 255) / 256, n_sys);
  k_gq_reduce<<<grid, 256, 0, s>>>(sinfo, sys_g0, sys_g1, gq, gb0, gb1, n_iw, mmax, first, acc);
  return cudaGetLastError();
}

cudaError_t launch_einf(const KInfo* kinfo, const SInfo* sinfo, const double2* H, const double2* P,
                        const double2* Sinf, int n_k, double2* Einf, double* trHE, cudaStream_t s) {
  k_einf<<<n_k, kThreads, 0, s>>>(kinfo, sinfo, H, P, Sinf, Einf, trHE);
  return cudaGetLastError();
}

cudaError_t launch_upcast(const float2* in, double2* out, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_upcast<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, out, n);
  return cudaGetLastError();
}

cudaError_t launch_diag_to_dense(const KInfo* kinfo, const double2* diag, const int64_t* offD,
                                 int n_k, double2* H, cudaStream_t s) {
  k_diag_to_dense<<<n_k, 256, 0, s>>>(kinfo, diag, offD, H);
  return cudaGetLastError();
}

cudaError_t launch_mubar_reduce(const KInfo* /*kinfo*/, const SInfo* sinfo, int n_sys, int n_chunks,
                                const double* mubar_part, double* out, cudaStream_t s) {
  k_mubar_reduce<<<n_sys, kThreads, 0, s>>>(sinfo, n_chunks, mubar_part, out);
  return cudaGetLastError();
}

}  // namespace gf

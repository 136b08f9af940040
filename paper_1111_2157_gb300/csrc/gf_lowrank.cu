// Low-rank (eigenbasis) point kernel of the lattice Green's function (sm_103a).
//
// With H_k = U diag(eps) U^+ (one Hermitian eigenproblem per k, computed once
// per Hamiltonian by k_lr_setup in gf_eig.cu) and Pt = P_k U, the inverse of
// Eq. dmftloop1 is, in the eigenbasis (Woodbury identity),
//   U^+ G U = D + D Pt^+ K Pt D,   D = diag(1 / (i w_n + mu - eps)),
//   K = M^{-1} Sigma,  M = I - Sigma g0,  g_j = Pt D^{j+1} Pt^+  (m x m),
// so every output of the point kernel follows from m x m algebra:
//   Tr G    = sum_b d_b + Tr(K g1)
//   Tr G^2  = sum_b d_b^2 + 2 Tr(K g2) + Tr(K g1 K g1)
//   P G P^+ = g0 + g0 K g0                                   (G_loc, A_k)
//   P G^2 P^+ = g1 + g1 K g0 + g0 K g1 + g0 K g1 K g0         (B_k)
//   U^+ G U (for rho_k) = D + D Pt^+ (K Pt) D, accumulated in the eigenbasis
//   and rotated back once per k by k_lr_rotate.
// Work per point: 3 N_b m^2 + O(m^3) complex multiply-adds instead of N_b^3;
// the partial sums have exactly the layout of k_point_fp64's, so the same
// finalize and reduction kernels consume them.
#include <math.h>
#include <stdint.h>

#include "gf_complex.cuh"
#include "gf_internal.cuh"
#include "gf_pair.cuh"

namespace gf {

namespace {

using namespace cx;




__device__ __forceinline__ double lr_block_sum(double v, double* red) {
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

// Gauss-Jordan reduction of the M x 2M augmented matrix [M_ | Sigma] (row-major,
// leading dimension 2M) to [I | M_^{-1} Sigma], partial pivoting on the left
// block.  col and urow: 2M complex scratch each.
__device__ void gj_augmented(double2* aug, int M, double2* col, double2* urow, int* status) {
  __shared__ int s_p;
  __shared__ double2 s_r;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int W = 2 * M;
  for (int j = 0; j < M; ++j) {
    if (warp == 0) {
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
      if (lane == 0) {
        if (best == 0ULL || best >= 0x7ff0000000000000ULL) atomicOr(status, kFlagSingular);
        s_p = bi;
        s_r = crcp(aug[bi * W + j]);
      }
    }
    __syncthreads();
    const int pr = s_p;
    const double2 r = s_r;
    for (int c = tid; c < W; c += kThreads) {
      const double2 vp = aug[pr * W + c];
      urow[c] = (c == j) ? make_double2(1.0, 0.0) : cmul(vp, r);
      if (pr != j) aug[pr * W + c] = aug[j * W + c];
    }
    for (int i = tid; i < M; i += kThreads) col[i] = (i == pr) ? aug[j * W + j] : aug[i * W + j];
    __syncthreads();
    // columns c < j of the left block are unit columns already: nothing to update
    const int Wj = W - j;
    for (int e = tid; e < M * Wj; e += kThreads) {
      const int i = e / Wj, c = j + (e - (e / Wj) * Wj);
      if (i == j) {
        aug[i * W + c] = urow[c];
      } else if (c == j) {
        aug[i * W + c] = make_double2(0.0, 0.0);
      } else {
        const double2 l = col[i], u = urow[c];
        double2 v = aug[i * W + c];
        v.x = fma(-l.x, u.x, fma(l.y, u.y, v.x));
        v.y = fma(-l.x, u.y, fma(-l.y, u.x, v.y));
        aug[i * W + c] = v;
      }
    }
    __syncthreads();
  }
}

// C = X Y for M x M matrices (X with leading dimension ldx), all threads.
__device__ __forceinline__ void mm(double2* C, const double2* X, int ldx, const double2* Y, int M) {
  for (int e = threadIdx.x; e < M * M; e += kThreads) {
    const int a = e / M, b = e - (e / M) * M;
    double2 acc = make_double2(0.0, 0.0);
    for (int c = 0; c < M; ++c) cmac(acc, X[a * ldx + c], Y[c * M + b]);
    C[e] = acc;
  }
}

// Complex FP32 pairs: c = (re, im) as float4 (re.h, re.l, im.h, im.l).
__device__ __forceinline__ void cp_mac(pair::f2& re, pair::f2& im, float4 a, float4 b) {
  using pair::f2;
  const f2 ar{a.x, a.y}, ai{a.z, a.w}, br{b.x, b.y}, bi{b.z, b.w};
  pair::mac(re, ar, br);
  pair::mac(re, f2{-ai.h, -ai.l}, bi);
  pair::mac(im, ar, bi);
  pair::mac(im, ai, br);
}
__device__ __forceinline__ float4 cp_pack(pair::f2 re, pair::f2 im) {
  float s, e;
  pair::two_sum(re.h, re.l, s, e);  // renormalise: |lo| <= ulp(hi) / 2
  re = pair::f2{s, e};
  pair::two_sum(im.h, im.l, s, e);
  im = pair::f2{s, e};
  return make_float4(re.h, re.l, im.h, im.l);
}
__device__ __forceinline__ unsigned pivot_key_p(float4 a) {
  const unsigned r = __float_as_uint(a.x) & 0x7fffffffu, i = __float_as_uint(a.z) & 0x7fffffffu;
  return r > i ? r : i;
}

// [I - Sigma g0 | Sigma] in FP32 pairs, reduced by Gauss-Jordan with partial
// pivoting (key from the head words) to [I | K], then K converted to FP64 in
// place: the float4 pairs and the double2 values have the same size, and each
// thread converts the entries it owns.  Sp, g0p: M x M pairs; augp aliases aug.
__device__ void pair_solve(const float4* Sp, const float4* g0p, double2* aug, int M, float4* colp,
                           float4* urowp, int* status) {
  using pair::f2;
  __shared__ int s_p;
  __shared__ float4 s_r;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int W = 2 * M;
  float4* augp = reinterpret_cast<float4*>(aug);
  for (int e = tid; e < M * M; e += kThreads) {
    const int a = e / M, c = e - (e / M) * M;
    f2 re{a == c ? 1.f : 0.f, 0.f}, im{0.f, 0.f};
    for (int x = 0; x < M; ++x) {
      const float4 sv = Sp[a * M + x];
      cp_mac(re, im, make_float4(-sv.x, -sv.y, -sv.z, -sv.w), g0p[x * M + c]);
    }
    augp[a * W + c] = cp_pack(re, im);
    augp[a * W + M + c] = Sp[e];
  }
  __syncthreads();
  for (int j = 0; j < M; ++j) {
    if (warp == 0) {
      unsigned best = 0u;
      int bi = 0x7fffffff;
      for (int i = j + lane; i < M; i += 32) {
        const unsigned key = pivot_key_p(augp[i * W + j]);
        if (bi == 0x7fffffff || key > best) { best = key; bi = i; }
      }
      for (int off = 16; off; off >>= 1) {
        const unsigned ob = __shfl_xor_sync(0xffffffffu, best, off);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (lane == 0) {
        if (best == 0u || best >= 0x7f800000u) atomicOr(status, kFlagSingular);
        s_p = bi;
        // reciprocal of the pivot in FP64 (one per step), split into pairs
        const float4 pv = augp[bi * W + j];
        const double2 r = crcp(make_double2((double)pv.x + (double)pv.y, (double)pv.z + (double)pv.w));
        const f2 rr = pair::split(r.x), ri = pair::split(r.y);
        s_r = make_float4(rr.h, rr.l, ri.h, ri.l);
      }
    }
    __syncthreads();
    const int pr = s_p;
    const float4 r = s_r;
    for (int c = tid; c < W; c += kThreads) {
      const float4 vp = augp[pr * W + c];
      if (c == j) {
        urowp[c] = make_float4(1.f, 0.f, 0.f, 0.f);
      } else {
        f2 re{0.f, 0.f}, im{0.f, 0.f};
        cp_mac(re, im, vp, r);
        urowp[c] = cp_pack(re, im);
      }
      if (pr != j) augp[pr * W + c] = augp[j * W + c];
    }
    for (int i = tid; i < M; i += kThreads) colp[i] = (i == pr) ? augp[j * W + j] : augp[i * W + j];
    __syncthreads();
    const int Wj = W - j;
    for (int e = tid; e < M * Wj; e += kThreads) {
      const int i = e / Wj, c = j + (e - (e / Wj) * Wj);
      if (i == j) {
        augp[i * W + c] = urowp[c];
      } else if (c == j) {
        augp[i * W + c] = make_float4(0.f, 0.f, 0.f, 0.f);
      } else {
        const float4 v = augp[i * W + c], l = colp[i];
        f2 re{v.x, v.y}, im{v.z, v.w};
        cp_mac(re, im, make_float4(-l.x, -l.y, -l.z, -l.w), urowp[c]);
        augp[i * W + c] = cp_pack(re, im);
      }
    }
    __syncthreads();
  }
  // K (right half) to FP64 in place; the left half (the identity) is not read again
  for (int e = tid; e < M * M; e += kThreads) {
    const int a = e / M, c = e - (e / M) * M;
    const float4 v = augp[a * W + M + c];
    aug[a * W + M + c] = make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
  }
  __syncthreads();
}

// The band sums of g0, g1, g2 in FP32-pair arithmetic: the same pair loop as the
// FP64 path (pairs a <= c, S threads per pair, warp-uniform bound), with
// t = Pt_a conj(Pt_c) and the d^j as pairs; results converted to FP64.
__device__ __forceinline__ void pair_band_sums(int NP, int S, int M, int N, bool need_g1,
                                               bool need_g2, int t_in_smem, const float4* sPtd,
                                               const float4* sTpd, const float4* sDd, double2* g0,
                                               double2* g1, double2* g2, float4* g0p) {
  using pair::f2;
  const int tid = threadIdx.x;
  for (int base = 0; base < NP * S; base += kThreads) {
    const int e = base + tid;
    const bool valid = e < NP * S;
    const int pq = valid ? e / S : 0, part = valid ? e - (e / S) * S : 0;
    int a = 0, rem = pq;
    while (rem >= M - a) { rem -= M - a; ++a; }
    const int c = a + rem;
    // x[j][0..3]: (Xr.re, Xr.im, Xi.re, Xi.im) of g_j
    f2 x[3][4];
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) x[j][q] = f2{0.f, 0.f};
    for (int b = part; valid && b < N; b += S) {
      f2 tr, ti;
      if (t_in_smem) {
        const float4 t4 = sTpd[pq * N + b];
        tr = f2{t4.x, t4.y};
        ti = f2{t4.z, t4.w};
      } else {
        // t = Pt_a conj(Pt_c): re = ar cr + ai ci, im = ai cr - ar ci
        const float4 u = sPtd[a * N + b], v = sPtd[c * N + b];
        const f2 ar{u.x, u.y}, ai{u.z, u.w}, cr{v.x, v.y}, ci{v.z, v.w};
        tr = f2{0.f, 0.f};
        ti = f2{0.f, 0.f};
        pair::mac(tr, ar, cr);
        pair::mac(tr, ai, ci);
        pair::mac(ti, ai, cr);
        pair::mac(ti, f2{-ar.h, -ar.l}, ci);
      }
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        if ((j == 1 && !need_g1) || (j == 2 && !need_g2)) continue;
        const float4 d4 = sDd[j * N + b];
        const f2 dr{d4.x, d4.y}, di{d4.z, d4.w};
        pair::mac(x[j][0], tr, dr);
        pair::mac(x[j][1], ti, dr);
        pair::mac(x[j][2], tr, di);
        pair::mac(x[j][3], ti, di);
      }
    }
    for (int off = 1; off < S; off <<= 1) {
#pragma unroll
      for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const f2 o{__shfl_xor_sync(0xffffffffu, x[j][q].h, off),
                     __shfl_xor_sync(0xffffffffu, x[j][q].l, off)};
          pair::add(x[j][q], o);
        }
    }
    if (valid && part == 0) {
      double2* gs[3] = {g0, g1, g2};
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const double xrr = pair::value(x[j][0]), xri = pair::value(x[j][1]);
        const double xir = pair::value(x[j][2]), xii = pair::value(x[j][3]);
        gs[j][a * M + c] = make_double2(xrr - xii, xri + xir);
        gs[j][c * M + a] = make_double2(xrr + xii, xir - xri);
      }
      // g0 also as pairs for the pair elimination: (g0)_ac = Xr + i Xi, (g0)_ca = conj(Xr) + i conj(Xi)
      const f2 rr = x[0][0], ri = x[0][1], ir = x[0][2], ii = x[0][3];
      f2 ac_re = rr, ac_im = ri, ca_re = rr, ca_im = ir;
      pair::add(ac_re, f2{-ii.h, -ii.l});
      pair::add(ac_im, ir);
      pair::add(ca_re, ii);
      pair::add(ca_im, f2{-ri.h, -ri.l});
      g0p[a * M + c] = make_float4(ac_re.h, ac_re.l, ac_im.h, ac_im.l);
      g0p[c * M + a] = make_float4(ca_re.h, ca_re.l, ca_im.h, ca_im.l);
    }
  }
}

// PAIR: the band sums of g0, g1, g2 in FP32-pair arithmetic (mixed precision);
// everything else in FP64.
template <bool PAIR>
__global__ void __launch_bounds__(kThreads) k_point_lr(const PointParams p, const LowRank lr) {
  extern __shared__ __align__(16) unsigned char smraw[];
  double2* sm = reinterpret_cast<double2*>(smraw);
  __shared__ int s_item;
  __shared__ double s_red[kThreads / 32];
  const LRLayout L = make_lr_layout(p.nbmax, p.mmax, p.mode, lr.t_in_smem, PAIR ? 1 : 0);
  double2* sPt = sm + L.offPt;
  double2* sD = sm + L.offD;  // d, d^2, d^3 per band
  double2* sS = sm + L.offS;
  double2* g0 = sm + L.offG;
  double2* g1 = g0 + p.mmax * p.mmax;
  double2* g2 = g1 + p.mmax * p.mmax;
  double2* aug = sm + L.offAug;
  double2* sC = sm + L.offC;    // K g1
  double2* sC2 = sm + L.offC2;  // K g0
  double2* sX = sm + L.offX;    // K Pt (rho) / A, B, Gbar, Gbar A^+ (adjoint)
  double2* sCol = sm + L.offCol;
  double2* sU = sm + L.offU;
  double2* sTp = sm + L.offT;
  float4* sPtd = reinterpret_cast<float4*>(sm + L.offPtd);  // (re.h, re.l, im.h, im.l)
  float4* sDd = reinterpret_cast<float4*>(sm + L.offDd);
  float4* sTpd = reinterpret_cast<float4*>(sTp);             // pair table (PAIR)
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
      const int N = ki.nb, M = si.m, W = 2 * M;
      const double mu = p.mu[ki.sys];
      const double beta = si.beta;
      const double wk = ki.w;
      const double* eps = lr.eps + lr.offD[kk];
      double nbar = 0.0;
      if ((p.mode & kAdj) && p.nbar) nbar = p.nbar[ki.sys];
      for (int e = tid; e < M * N; e += kThreads) sPt[e] = lr.Pt[ki.offP + e];
      // pairs a <= c, enumerated row by row; S threads share one pair's band sum
      const int NP = M * (M + 1) / 2;
      const int S = NP >= kThreads ? 1 : (2 * NP <= kThreads ? (4 * NP <= kThreads ? 4 : 2) : 1);
      if (PAIR) {
        for (int e = tid; e < M * N; e += kThreads) {
          const double2 v = lr.Pt[ki.offP + e];
          const pair::f2 re = pair::split(v.x), im = pair::split(v.y);
          sPtd[e] = make_float4(re.h, re.l, im.h, im.l);
        }
      }
      if (lr.t_in_smem) {
        __syncthreads();
        for (int e = tid; e < NP * N; e += kThreads) {
          const int pq = e / N, b = e - (e / N) * N;
          int a = 0, rem = pq;
          while (rem >= M - a) { rem -= M - a; ++a; }
          const int c = a + rem;
          double2 t = make_double2(0.0, 0.0);
          cmac_cb(t, sPt[a * N + b], sPt[c * N + b]);
          if (PAIR) {
            const pair::f2 re = pair::split(t.x), im = pair::split(t.y);
            sTpd[e] = make_float4(re.h, re.l, im.h, im.l);
          } else {
            sTp[e] = t;
          }
        }
      }
      double acc_tr = 0.0, acc_g2 = 0.0, acc_mu = 0.0;
      for (int n = it.n0; n < it.n1; ++n) {
        const double wn = (2.0 * n + 1.0) * M_PI / beta;
        const double2* Sg = p.Sig + si.offSig + (int64_t)n * M * M;
        __syncthreads();
        for (int b = tid; b < N; b += kThreads) {
          // d = 1 / (x + i w) = (x - i w) / (x^2 + w^2), x = mu - eps_b
          const double x = mu - eps[b];
          const double q = 1.0 / fma(x, x, wn * wn);
          const double2 d = make_double2(x * q, -wn * q);
          const double2 d2 = cmul(d, d);
          sD[b] = d;
          sD[N + b] = d2;
          sD[2 * N + b] = cmul(d2, d);
          if (PAIR) {
            const double2 d3 = sD[2 * N + b];
            const double2 dd[3] = {d, d2, d3};
  #pragma unroll
            for (int j = 0; j < 3; ++j) {
              const pair::f2 re = pair::split(dd[j].x), im = pair::split(dd[j].y);
              sDd[j * N + b] = make_float4(re.h, re.l, im.h, im.l);
            }
          }
        }
        for (int e = tid; e < M * M; e += kThreads) sS[e] = Sg[e];
        __syncthreads();
        // g_j = Pt D^{j+1} Pt^+.  With d = dr + i di and t = Pt_ab conj(Pt_cb):
        // (g_j)_ac = Xr + i Xi and (g_j)_ca = conj(Xr) + i conj(Xi), Xr = sum t dr,
        // Xi = sum t di, so only the pairs a <= c are summed.
        const bool need_g2 = (p.mode & kOcc) != 0;
        const bool need_g1 = (p.mode & (kOcc | kAdj)) != 0;
        // (the loop bound is uniform across the block, so every lane of a warp reaches the
        // shuffles; lanes past the end sum nothing and write nothing)
        if (PAIR) {
          pair_band_sums(NP, S, M, N, need_g1, need_g2, lr.t_in_smem, sPtd, sTpd, sDd, g0, g1, g2,
                         reinterpret_cast<float4*>(sC));
        } else
        for (int base = 0; base < NP * S; base += kThreads) {
          const int e = base + tid;
          const bool valid = e < NP * S;
          const int pq = valid ? e / S : 0, part = valid ? e - (e / S) * S : 0;
          int a = 0, rem = pq;
          while (rem >= M - a) { rem -= M - a; ++a; }
          const int c = a + rem;
          double2 xr0 = make_double2(0.0, 0.0), xi0 = xr0, xr1 = xr0, xi1 = xr0, xr2 = xr0, xi2 = xr0;
          for (int b = part; valid && b < N; b += S) {
            double2 t;
            if (lr.t_in_smem) {
              t = sTp[pq * N + b];
            } else {
              t = make_double2(0.0, 0.0);
              cmac_cb(t, sPt[a * N + b], sPt[c * N + b]);
            }
            const double2 d0 = sD[b];
            xr0.x = fma(t.x, d0.x, xr0.x); xr0.y = fma(t.y, d0.x, xr0.y);
            xi0.x = fma(t.x, d0.y, xi0.x); xi0.y = fma(t.y, d0.y, xi0.y);
            if (need_g1) {
              const double2 d1 = sD[N + b];
              xr1.x = fma(t.x, d1.x, xr1.x); xr1.y = fma(t.y, d1.x, xr1.y);
              xi1.x = fma(t.x, d1.y, xi1.x); xi1.y = fma(t.y, d1.y, xi1.y);
            }
            if (need_g2) {
              const double2 d2 = sD[2 * N + b];
              xr2.x = fma(t.x, d2.x, xr2.x); xr2.y = fma(t.y, d2.x, xr2.y);
              xi2.x = fma(t.x, d2.y, xi2.x); xi2.y = fma(t.y, d2.y, xi2.y);
            }
          }
          // the S partial sums of a pair sit in consecutive lanes of one warp (S | 32 and
          // base is a multiple of 32)
          for (int off = 1; off < S; off <<= 1) {
  #define GF_LR_RED(v)                                        \
    v.x += __shfl_xor_sync(0xffffffffu, v.x, off);            \
    v.y += __shfl_xor_sync(0xffffffffu, v.y, off);
            GF_LR_RED(xr0) GF_LR_RED(xi0) GF_LR_RED(xr1) GF_LR_RED(xi1) GF_LR_RED(xr2) GF_LR_RED(xi2)
  #undef GF_LR_RED
          }
          if (valid && part == 0) {
            g0[a * M + c] = make_double2(xr0.x - xi0.y, xr0.y + xi0.x);
            g0[c * M + a] = make_double2(xr0.x + xi0.y, xi0.x - xr0.y);
            g1[a * M + c] = make_double2(xr1.x - xi1.y, xr1.y + xi1.x);
            g1[c * M + a] = make_double2(xr1.x + xi1.y, xi1.x - xr1.y);
            g2[a * M + c] = make_double2(xr2.x - xi2.y, xr2.y + xi2.x);
            g2[c * M + a] = make_double2(xr2.x + xi2.y, xi2.x - xr2.y);
          }
        }
        __syncthreads();
        if (PAIR) {
          // Sigma as pairs in sC2's storage (sC holds g0 as pairs); both are free until K exists
          float4* Sp = reinterpret_cast<float4*>(sC2);
          for (int e = tid; e < M * M; e += kThreads) {
            const pair::f2 re = pair::split(sS[e].x), im = pair::split(sS[e].y);
            Sp[e] = make_float4(re.h, re.l, im.h, im.l);
          }
          __syncthreads();
          pair_solve(Sp, reinterpret_cast<const float4*>(sC), aug, M, reinterpret_cast<float4*>(sCol),
                     reinterpret_cast<float4*>(sU), p.status);
        } else {
          // aug = [I - Sigma g0 | Sigma]
          for (int e = tid; e < M * M; e += kThreads) {
            const int a = e / M, c = e - (e / M) * M;
            double2 acc = make_double2(a == c ? 1.0 : 0.0, 0.0);
            for (int x = 0; x < M; ++x) {
              const double2 s = sS[a * M + x], g = g0[x * M + c];
              acc.x -= fma(s.x, g.x, -s.y * g.y);
              acc.y -= fma(s.x, g.y, s.y * g.x);
            }
            aug[a * W + c] = acc;
            aug[a * W + M + c] = sS[e];
          }
          __syncthreads();
          gj_augmented(aug, M, sCol, sU, p.status);
        }
        const double2* K = aug + M;  // K[a * W + c]
        if (p.mode & (kOcc | kAdj)) mm(sC, K, W, g1, M);
        if (p.mode & (kGloc | kAdj)) mm(sC2, K, W, g0, M);
        __syncthreads();
        if (p.mode & kOcc) {
          for (int b = tid; b < N; b += kThreads) {
            acc_tr += sD[b].x;
            acc_g2 += sD[N + b].x;
          }
          for (int e = tid; e < M * M; e += kThreads) {
            const int a = e / M, c = e - (e / M) * M;
            // Re of K_ac g1_ca, 2 K_ac g2_ca and (K g1)_ac (K g1)_ca
            const double2 kk = K[a * W + c];
            const double2 u = g1[c * M + a], v = g2[c * M + a];
            const double2 x = sC[e], y = sC[c * M + a];
            acc_tr += fma(kk.x, u.x, -kk.y * u.y);
            acc_g2 += 2.0 * fma(kk.x, v.x, -kk.y * v.y) + fma(x.x, y.x, -x.y * y.y);
          }
        }
        if (p.mode & kRho) {
          // X = K Pt (M x N), then S' += D + D Pt^+ X D in the eigenbasis
          for (int e = tid; e < M * N; e += kThreads) {
            const int a = e / N, b = e - (e / N) * N;
            double2 acc = make_double2(0.0, 0.0);
            for (int c = 0; c < M; ++c) cmac(acc, K[a * W + c], sPt[c * N + b]);
            sX[e] = acc;
          }
          __syncthreads();
          double2* S = p.rho_part + (int64_t)it.chunk * p.rho_chunk_stride + ki.offH;
          const bool first = (n == it.n0);
          for (int e = tid; e < N * N; e += kThreads) {
            const int b = e / N, c = e - (e / N) * N;
            double2 acc = make_double2(0.0, 0.0);
            for (int a = 0; a < M; ++a) cmac_ca(acc, sPt[a * N + b], sX[a * N + c]);
            double2 g = cmul(cmul(sD[b], acc), sD[c]);
            if (b == c) { g.x += sD[b].x; g.y += sD[b].y; }
            if (first) {
              S[e] = g;
            } else {
              double2 s = S[e];
              s.x += g.x; s.y += g.y;
              S[e] = s;
            }
          }
        }
        if (p.mode & kGloc) {
          // P G P^+ = g0 + g0 (K g0)
          double2* out = p.gq + ((int64_t)(it.g - p.gb0) * p.n_iw + n) * p.mmax * p.mmax;
          for (int e = tid; e < M * M; e += kThreads) {
            const int a = e / M, c = e - (e / M) * M;
            double2 acc = g0[e];
            for (int x = 0; x < M; ++x) cmac(acc, g0[a * M + x], sC2[x * M + c]);
            gq_put(&out[e], q, make_double2(wk * acc.x, wk * acc.y));
          }
        }
        if (p.mode & kAdj) {
          double2* Aq = sX;
          double2* Bq = sX + M * M;
          double2* Gb = sX + 2 * M * M;
          double2* Mt = sX + 3 * M * M;
          double2* CC2 = aug;  // K no longer needed: (K g1)(K g0) in the left half of aug
          __syncthreads();
          for (int e = tid; e < M * M; e += kThreads) {
            const int a = e / M, c = e - (e / M) * M;
            double2 acc = make_double2(0.0, 0.0);
            for (int x = 0; x < M; ++x) cmac(acc, sC[a * M + x], sC2[x * M + c]);
            CC2[a * W + c] = acc;
          }
          __syncthreads();
          // A = g0 + g0 C2;  B = g1 + g1 C2 + g0 (C + C C2)
          for (int e = tid; e < M * M; e += kThreads) {
            const int a = e / M, c = e - (e / M) * M;
            double2 aa = g0[e], bb = g1[e];
            for (int x = 0; x < M; ++x) {
              const double2 c2 = sC2[x * M + c];
              cmac(aa, g0[a * M + x], c2);
              cmac(bb, g1[a * M + x], c2);
              double2 t = sC[x * M + c];
              const double2 u = CC2[x * W + c];
              t.x += u.x;
              t.y += u.y;
              cmac(bb, g0[a * M + x], t);
            }
            Aq[e] = aa;
            Bq[e] = bb;
          }
          __syncthreads();
          const bool have_gbar = (p.gbar != nullptr);
          if (have_gbar) {
            const double2* Gsrc = p.gbar + si.offSig + (int64_t)n * M * M;
            for (int e = tid; e < M * M; e += kThreads) Gb[e] = Gsrc[e];
            __syncthreads();
            for (int e = tid; e < M * M; e += kThreads) {
              const int a = e / M, b = e - (e / M) * M;
              double2 acc = make_double2(0.0, 0.0);
              for (int c = 0; c < M; ++c) cmac_cb(acc, Gb[a * M + c], Aq[b * M + c]);
              Mt[e] = acc;
            }
            __syncthreads();
            for (int e = tid; e < M * M; e += kThreads) {
              const double2 g = Gb[e], b = Bq[e];
              acc_mu -= wk * fma(g.x, b.x, g.y * b.y);
            }
          }
          double2* out = p.gq + ((int64_t)(it.g - p.gb0) * p.n_iw + n) * p.mmax * p.mmax;
          const double cb = nbar * 2.0 / beta;
          for (int e = tid; e < M * M; e += kThreads) {
            const int a = e / M, b = e - (e / M) * M;
            double2 acc = make_double2(0.0, 0.0);
            if (have_gbar)
              for (int c = 0; c < M; ++c) cmac_ca(acc, Aq[c * M + a], Mt[c * M + b]);
            const double2 bt = Bq[b * M + a];
            acc.x = fma(cb, bt.x, acc.x);
            acc.y = fma(-cb, bt.y, acc.y);
            gq_put(&out[e], q, make_double2(wk * acc.x, wk * acc.y));
          }
        }
      }
      if (p.mode & kOcc) {
        const double tr = lr_block_sum(acc_tr, s_red);
        const double g2s = lr_block_sum(acc_g2, s_red);
        if (tid == 0) {
          double* o = p.occ_part + ((int64_t)kk * p.n_chunks + it.chunk) * 2;
          o[0] = tr;
          o[1] = g2s;
        }
      }
      if (p.mode & kAdj) {
        const double mb = lr_block_sum(acc_mu, s_red);
        if (tid == 0) p.mubar_part[(int64_t)kk * p.n_chunks + it.chunk] = mb;
      }
      __syncthreads();
    }
  }
}

// rho_part chunk 0 <- U (sum_c S'_c) U^+ for every k (one CTA per k); T is a
// scratch of the size of H.
__global__ void __launch_bounds__(kThreads)
    k_lr_rotate(const KInfo* __restrict__ kinfo, const double2* __restrict__ U, double2* rho_part,
                int64_t stride, int n_chunks, double2* T) {
  const KInfo ki = kinfo[blockIdx.x];
  const int N = ki.nb;
  const double2* Uk = U + ki.offH;
  double2* S0 = rho_part + ki.offH;
  double2* Tk = T + ki.offH;
  // T = (sum_c S'_c) U^+
  for (int e = threadIdx.x; e < N * N; e += kThreads) {
    const int i = e / N, j = e - (e / N) * N;
    double2 acc = make_double2(0.0, 0.0);
    for (int l = 0; l < N; ++l) {
      double2 s = make_double2(0.0, 0.0);
      for (int c = 0; c < n_chunks; ++c) {
        const double2 v = rho_part[(int64_t)c * stride + ki.offH + i * N + l];
        s.x += v.x;
        s.y += v.y;
      }
      cmac_cb(acc, s, Uk[j * N + l]);
    }
    Tk[e] = acc;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < N * N; e += kThreads) {
    const int i = e / N, j = e - (e / N) * N;
    double2 acc = make_double2(0.0, 0.0);
    for (int l = 0; l < N; ++l) cmac(acc, Uk[i * N + l], Tk[l * N + j]);
    S0[e] = acc;
  }
}

}  // namespace

size_t point_lr_smem(int nbmax, int mmax, int mode, int t_in_smem, int pair_sums) {
  return make_lr_layout(nbmax, mmax, mode, t_in_smem, pair_sums).bytes;
}

int point_lr_blocks_per_sm(size_t smem, int pair_sums) {
  int n = 0;
  if (pair_sums) {
    cudaFuncSetAttribute(k_point_lr<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_point_lr<true>, kThreads, smem);
  } else {
    cudaFuncSetAttribute(k_point_lr<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_point_lr<false>, kThreads, smem);
  }
  return n;
}

cudaError_t launch_point_lr(const PointParams& p, const LowRank& lr, int grid, size_t smem,
                            cudaStream_t s) {
  cudaError_t e;
  if (lr.pair_sums) {
    e = cudaFuncSetAttribute(k_point_lr<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_point_lr<true><<<grid, kThreads, smem, s>>>(p, lr);
  } else {
    e = cudaFuncSetAttribute(k_point_lr<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_point_lr<false><<<grid, kThreads, smem, s>>>(p, lr);
  }
  return cudaGetLastError();
}

cudaError_t launch_lr_rotate(const KInfo* kinfo, int n_k, const double2* U, double2* rho_part,
                             int64_t stride, int n_chunks, double2* T, cudaStream_t s) {
  k_lr_rotate<<<n_k, kThreads, 0, s>>>(kinfo, U, rho_part, stride, n_chunks, T);
  return cudaGetLastError();
}

}  // namespace gf

// Mixed-precision point kernel of the lattice Green's function path (sm_103a):
// single-word FP32 Gauss-Jordan inverse held in registers, FP64 Matsubara sums,
// and one step of iterative refinement, with an FP32-pair residual, of the
// columns of G that the projections consume.
//
// Arithmetic per (k, i w_n) point:
//   1. A = (i w_n + mu) I - H_k - P_k^+ (Sigma(i w_n) P_k)  in FP32 (Eq. dmftloop1);
//      the diagonal mu - H_ii is formed in FP64 and rounded once.
//   2. X = A^{-1} by Gauss-Jordan elimination with partial pivoting in FP32.
//      On GB300 one SM issues 128 FP32 FMAs per clock against 2 FP64 FMAs, so
//      this costs about 1/64 of the FP64 inverse; its error is about
//      kappa(A) * 2^-24 relative per entry.
//   3. Epilogues:
//      kOcc  Re Tr X and Re Tr X^2, summed over the frequencies in FP64    -> N, dN/dmu
//      kRho  S_k += X in FP64                                             -> rho_k
//      kGloc Y = X P^+ refined once: R = P^+ - A Y in FP32 pairs (A from the
//            FP32-pair copies of H, P and Sigma), Y += X R in FP32; then
//            w_k P Y with P Y0 in pairs                                   -> G_loc
//      kAdj  the same refinement of Z = P X (R' = P - Z A), then A_k = P Y,
//            B_k = Z Y and w_k [A^+ Gbar A^+ + nbar (2/beta) B^+] in pairs
// One refinement step leaves an error of about (kappa 2^-24)^2 plus the pair
// residual's 2^-44 kappa, far below the FP32 inverse's own, for the m
// columns that G_loc and the adjoint use (m << N_b), at 2 N_b^2 m extra
// multiply-adds instead of the N_b^3 of refining the whole inverse.
//
// Thread layout: the CTA is warp 0 (pivot lookahead) plus a TR x TC grid of
// owners; owner (tr, tc) holds the RA x RB entries (tr + TR a, tc + TC b) of A
// in registers.  A pivot step reads RA multipliers and RB pivot-row entries
// from shared memory (broadcast) for RA RB register updates; warp 0 updates the
// next column, searches its pivot and forms the reciprocal meanwhile (one pivot
// of lookahead, two barriers per pivot).  After the inverse the tile is written
// once to shared memory (columns permuted by the pivot sequence) for the
// epilogues.
#include <math.h>
#include <stdint.h>

#include "gf_complex.cuh"
#include "gf_internal.cuh"
#include "gf_warp_gj.cuh"

namespace gf {

namespace {

using namespace cx;

constexpr int kMaxWarpsF = 24;

__device__ __forceinline__ double block_sum_f(double v, double* red) {
  // Deterministic: fixed xor tree in each warp, then warp 0 over the warps.
  for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double r = 0.0;
  if (warp == 0) {
    r = lane < nw ? red[lane] : 0.0;
    for (int off = 16; off; off >>= 1) r += __shfl_xor_sync(0xffffffffu, r, off);
  }
  return r;
}

__device__ __forceinline__ float2 f2zero() { return make_float2(0.f, 0.f); }
__device__ __forceinline__ float2 fneg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ cf conj_cf(const cf& a) { return cf{a.rh, a.rl, -a.ih, -a.il}; }
// Pivot key with the row index in its low 7 bits (rows < 128): the largest key
// wins, ties (and keys equal to 2^-16 relative) go to the lowest row.
__device__ __forceinline__ unsigned pack_key(float2 v, int i) {
  return (pivot_key_s(v) & ~127u) | (unsigned)(127 - i);
}
__device__ __forceinline__ float2 round_cf(const cf& a) {
  return make_float2(__fadd_rn(a.rh, a.rl), __fadd_rn(a.ih, a.il));
}


__device__ __forceinline__ float2 fconj(float2 a) { return make_float2(a.x, -a.y); }
// pair += single: q = q + d with d much smaller than q
__device__ __forceinline__ void add_single(cf& q, float2 d) {
  float s, t;
  two_sum(q.rh, d.x, s, t);
  q.rh = s;
  q.rl = __fadd_rn(q.rl, t);
  two_sum(q.ih, d.y, s, t);
  q.ih = s;
  q.il = __fadd_rn(q.il, t);
  cnorm(q);
}
// acc += a b for pair or single-word operands (single words enter exactly)
__device__ __forceinline__ void pmac(cf& acc, const cf& a, float2 b) { cacc1(acc, a, b); }
__device__ __forceinline__ void pmac(cf& acc, float2 a, const cf& b) { cacc1(acc, b, a); }
__device__ __forceinline__ void pmac(cf& acc, const cf& a, const cf& b) { cacc(acc, a, b); }
__device__ __forceinline__ void pmac(cf& acc, float2 a, float2 b) { cacc1(acc, cf{a.x, 0.f, a.y, 0.f}, b); }

// C (R x C) = sum_k la(r, k) lb(k, c) in FP32; each thread computes 2 x 2 blocks
// (two loaded values of each operand feed four multiply-adds).
template <class LA, class LB, class ST>
__device__ __forceinline__ void mm_f32(int R, int C, int K, LA la, LB lb, ST st) {
  const int cb = (C + 1) >> 1, nw = ((R + 1) >> 1) * cb;
  for (int w = threadIdx.x; w < nw; w += blockDim.x) {
    const int r0 = (w / cb) * 2, c0 = (w - (w / cb) * cb) * 2;
    const int r1 = min(r0 + 1, R - 1), c1 = min(c0 + 1, C - 1);
    float2 a00 = f2zero(), a01 = f2zero(), a10 = f2zero(), a11 = f2zero();
    for (int k = 0; k < K; ++k) {
      const float2 x0 = la(r0, k), x1 = la(r1, k), y0 = lb(k, c0), y1 = lb(k, c1);
      fmac(a00, x0, y0);
      fmac(a01, x0, y1);
      fmac(a10, x1, y0);
      fmac(a11, x1, y1);
    }
    st(r0, c0, a00);
    if (c1 != c0) st(r0, c1, a01);
    if (r1 != r0) {
      st(r1, c0, a10);
      if (c1 != c0) st(r1, c1, a11);
    }
  }
}

// C (R x C) = init(r, c) + sum_k la(r, k) lb(k, c) in FP32 pairs (operands pairs or
// single words), 2 x 2 blocks per
// thread; with S > 1 the k range is split in S parts whose partial sums go to
// part[S][R][C] (pairs) and are added in part order (deterministic).  The
// caller separates consecutive calls with a barrier; the function has its own
// barrier only when S > 1.
template <class LA, class LB, class IN, class ST>
__device__ __forceinline__ void mm_pair(int R, int C, int K, int S, float4* part, LA la, LB lb, IN init,
                                        ST st) {
  const int cb = (C + 1) >> 1, nb = ((R + 1) >> 1) * cb, nw = nb * S;
  const int kc = (K + S - 1) / S;
  for (int w = threadIdx.x; w < nw; w += blockDim.x) {
    const int blk = w / S, sp = w - blk * S;
    const int r0 = (blk / cb) * 2, c0 = (blk - (blk / cb) * cb) * 2;
    const int r1 = min(r0 + 1, R - 1), c1 = min(c0 + 1, C - 1);
    cf a00 = czero(), a01 = czero(), a10 = czero(), a11 = czero();
    const int k0 = sp * kc, k1 = min(K, k0 + kc);
    for (int k = k0; k < k1; ++k) {
      const auto x0 = la(r0, k), x1 = la(r1, k);
      const auto y0 = lb(k, c0), y1 = lb(k, c1);
      pmac(a00, x0, y0);
      pmac(a01, x0, y1);
      pmac(a10, x1, y0);
      pmac(a11, x1, y1);
      if (((k - k0) & 15) == 15) {
        cnorm(a00);
        cnorm(a01);
        cnorm(a10);
        cnorm(a11);
      }
    }
    cnorm(a00);
    cnorm(a01);
    cnorm(a10);
    cnorm(a11);
    if (S == 1) {
      auto fin = [&](int r, int c, cf v) {
        cf q = init(r, c);
        float s, t;
        two_sum(q.rh, v.rh, s, t);
        q.rh = s;
        q.rl = __fadd_rn(__fadd_rn(q.rl, v.rl), t);
        two_sum(q.ih, v.ih, s, t);
        q.ih = s;
        q.il = __fadd_rn(__fadd_rn(q.il, v.il), t);
        cnorm(q);
        st(r, c, q);
      };
      fin(r0, c0, a00);
      if (c1 != c0) fin(r0, c1, a01);
      if (r1 != r0) {
        fin(r1, c0, a10);
        if (c1 != c0) fin(r1, c1, a11);
      }
    } else {
      float4* pp = part + (size_t)sp * R * C;
      pp[r0 * C + c0] = st4(a00);
      if (c1 != c0) pp[r0 * C + c1] = st4(a01);
      if (r1 != r0) {
        pp[r1 * C + c0] = st4(a10);
        if (c1 != c0) pp[r1 * C + c1] = st4(a11);
      }
    }
  }
  if (S > 1) {
    __syncthreads();
    for (int e = threadIdx.x; e < R * C; e += blockDim.x) {
      const int r = e / C, c = e - r * C;
      cf q = init(r, c);
      for (int sp = 0; sp < S; ++sp) {
        const cf v = ld4(part[(size_t)sp * R * C + e]);
        float s, t;
        two_sum(q.rh, v.rh, s, t);
        q.rh = s;
        q.rl = __fadd_rn(__fadd_rn(q.rl, v.rl), t);
        two_sum(q.ih, v.ih, s, t);
        q.ih = s;
        q.il = __fadd_rn(__fadd_rn(q.il, v.il), t);
      }
      cnorm(q);
      st(r, c, q);
    }
  }
}
}  // namespace

// Shared-memory layout of k_point_f32r in bytes.  T = Sigma P (embedding) lives in
// the G region, which is free until the inverse is written there.
struct LayoutF {
  size_t oP, oS, oG, oT, oB, oD, oHii, oY0, oR, odY, oW, oV, oZ0, odZ, oQa, oQb, oMt, oPiv, bytes;
};

// Length of the pivot-step buffers: the register tiles cover TR RA and TC RB
// rows and columns, up to nbmax + 7 (RA, RB <= 8).
__host__ __device__ inline int f32r_nbp(int nbmax) { return nbmax + 8; }

__host__ __device__ inline LayoutF make_layout_f(int nbmax, int mmax, int mode) {
  LayoutF L;
  const size_t ld = (size_t)(nbmax | 1);
  const size_t mn = (size_t)mmax * nbmax, mm = (size_t)mmax * mmax;
  size_t o = 0;
  L.oP = o; o += 8 * mn;
  L.oS = o; o += 8 * mm;
  L.oG = o;
  size_t g = (size_t)nbmax * ld;
  if (g < mn) g = mn;
  if (g < mm) g = mm;
  o += 8 * g;
  L.oT = L.oG;
  L.oB = o; o += 8 * 6 * (size_t)f32r_nbp(nbmax);  // l, u, next column; two buffers each
  L.oD = o; o += 8 * (size_t)nbmax;                  // diagonal i w_n + mu - H_ii (FP32)
  o = (o + 15) & ~(size_t)15;
  L.oHii = o; o += 16 * (size_t)nbmax;               // H_ii (FP64)
  const bool refine = (mode & (kGloc | kAdj)) != 0;
  const bool adj = (mode & kAdj) != 0;
  auto take = [&o](size_t bytes) {  // 16-byte aligned region
    o = (o + 15) & ~(size_t)15;
    const size_t at = o;
    o += bytes;
    return at;
  };
  L.oW = take(refine ? 16 * mm : 0);   // P Y0 (pair), then Z0 P^+
  L.oV = take(refine ? 16 * mm : 0);   // Sigma (P Y0) (pair)
  L.oY0 = take(refine ? 8 * mn : 0);   // Y0 = X P^+ (N x m)
  L.oR = take(refine ? 8 * mn : 0);    // residual (N x m or m x N); with dY: partial sums
  L.odY = o; o += refine ? 8 * mn : 0; // X R (directly after R: 16 mn bytes together)
  L.oZ0 = take(adj ? 8 * mn : 0);      // Z0 = P X (m x N)
  L.odZ = take(adj ? 8 * mn : 0);      // R' X
  L.oQa = take(adj ? 16 * mm : 0);     // A_k = P Y (pair)
  L.oQb = take(adj ? 16 * mm : 0);     // B_k = Z Y (pair)
  L.oMt = take(adj ? 16 * mm : 0);     // Gbar A_k^+ (pair)
  o = (o + 15) & ~(size_t)15;
  L.oPiv = o; o += 3 * sizeof(int) * (size_t)nbmax;  // p, q = p^{-1}, row offsets
  L.bytes = o;
  return L;
}

namespace {

// Buffers of the refined-projection epilogues in shared memory (LayoutF).
struct EpiF {
  const float2* sP;                                // P_k in FP32 (M x N)
  float4 *sW, *sV, *sQa, *sQb, *sMt, *sPart;       // pairs
  float2 *sY0, *sR, *sdY, *sZ0, *sdZ;              // FP32
};

// The kRho, kGloc and kAdj epilogues of frequency n of k-point ki (slot q of the item's
// k-group), the inverse given as X[i][c] = sG[sRow[i] + sIdx[c]]; kRho adds X to the
// item's S_k, kGloc and kAdj refine G P^+ (and P G) once with an FP32-pair residual and
// store the k-group slot.  Every thread of the CTA runs it; consecutive products are
// separated by CTA barriers; the caller puts a barrier before (the inverse visible to
// all) and after (the buffers free).
__device__ __forceinline__ void f32r_epilogues(const PointParams& p, const EpiF& eb, const Item& it,
                                               const KInfo& ki, const SInfo& si, int q, int N, int M, int n,
                                               double wn, double mu, double beta, double wk, double nbar,
                                               const float4* Hkp, const float4* Pkp, const float2* sG,
                                               const int* sRow, const int* sIdx, double& acc_mu) {
  const int tid = threadIdx.x, nthr = blockDim.x;
  const float2* sP = eb.sP;
  float4 *sW = eb.sW, *sV = eb.sV, *sQa = eb.sQa, *sQb = eb.sQb, *sMt = eb.sMt, *sPart = eb.sPart;
  float2 *sY0 = eb.sY0, *sR = eb.sR, *sdY = eb.sdY, *sZ0 = eb.sZ0, *sdZ = eb.sdZ;
  if (p.mode & kRho) {
    double2* S = p.rho_part + (int64_t)it.chunk * p.rho_chunk_stride + ki.offH;
    const bool first = (n == it.n0);
    for (int e = tid; e < N * N; e += nthr) {
      const int i = e / N, c = e - i * N;
      const float2 g = sG[sRow[i] + sIdx[c]];
      if (first) {
        S[e] = make_double2((double)g.x, (double)g.y);
      } else {
        double2 s = S[e];
        s.x += (double)g.x;
        s.y += (double)g.y;
        S[e] = s;
      }
    }
  }
  if (p.mode & (kGloc | kAdj)) {
    const bool adj = (p.mode & kAdj) != 0;
    cf zw;  // -(i w_n + mu) as a pair
    split(-mu, zw.rh, zw.rl);
    split(-wn, zw.ih, zw.il);
    const float4* Sgp = p.Sd + si.offSig + (int64_t)n * M * M;
    auto X = [&](int i, int c) { return sG[sRow[i] + sIdx[c]]; };
    // Y0 = X P^+ (N x M)
    mm_f32(N, M, N, X, [&](int c, int b) { return fconj(sP[b * N + c]); },
           [&](int i, int b, float2 v) { sY0[i * M + b] = v; });
    // Z0 = P X (M x N)
    if (adj)
      mm_f32(M, N, N, [&](int a, int i) { return sP[a * N + i]; }, X,
             [&](int a, int c, float2 v) { sZ0[a * N + c] = v; });
    __syncthreads();
    // W = P Y0 (pairs; the sum over bands split in S parts, partials in the R region)
    const int S = max(1, min(4, N / M));
    mm_pair(M, M, N, S, sPart, [&](int a, int i) { return ld4(Pkp[a * N + i]); },
            [&](int i, int b) { return sY0[i * M + b]; }, [&](int, int) { return czero(); },
            [&](int a, int b, const cf& v) { sW[a * M + b] = st4(v); });
    __syncthreads();
    // V = Sigma W (pairs)
    mm_pair(M, M, M, 1, sPart, [&](int a, int x) { return ld4(Sgp[a * M + x]); },
            [&](int x, int b) { return ld4(sW[x * M + b]); }, [&](int, int) { return czero(); },
            [&](int a, int b, const cf& v) { sV[a * M + b] = st4(v); });
    __syncthreads();
    // R = P^+ - A Y0 = P^+ - (i w + mu) Y0 + H Y0 + P^+ V  (pairs, rounded to FP32)
    mm_pair(N, M, N, 1, sPart, [&](int i, int c) { return ld4(Hkp[i * N + c]); },
            [&](int c, int b) { return sY0[c * M + b]; },
            [&](int i, int b) {
              cf acc = conj_cf(ld4(Pkp[b * N + i]));
              cacc1(acc, zw, sY0[i * M + b]);
              for (int a = 0; a < M; ++a) cacc_ca(acc, ld4(Pkp[a * N + i]), ld4(sV[a * M + b]));
              return acc;
            },
            [&](int i, int b, const cf& v) { sR[i * M + b] = round_cf(v); });
    __syncthreads();
    // dY = X R (FP32);  Y = Y0 + dY
    mm_f32(N, M, N, X, [&](int c, int b) { return sR[c * M + b]; },
           [&](int i, int b, float2 v) { sdY[i * M + b] = v; });
    __syncthreads();
    // P Y = W + P dY (the second term in FP32)
    if (p.mode & kGloc) {
      double2* out = p.gq + ((int64_t)(it.g - p.gb0) * p.n_iw + n) * p.mmax * p.mmax;
      mm_f32(M, M, N, [&](int a, int i) { return sP[a * N + i]; },
             [&](int i, int b) { return sdY[i * M + b]; },
             [&](int a, int b, float2 d) {
               const double2 w = to_d2(ld4(sW[a * M + b]));
               gq_put(&out[a * M + b], q, make_double2(wk * (w.x + (double)d.x), wk * (w.y + (double)d.y)));
             });
    }
    if (adj) {
      // A_k = P Y in pairs
      mm_f32(M, M, N, [&](int a, int i) { return sP[a * N + i]; },
             [&](int i, int b) { return sdY[i * M + b]; },
             [&](int a, int b, float2 d) {
               cf q = ld4(sW[a * M + b]);
               add_single(q, d);
               sQa[a * M + b] = st4(q);
             });
      __syncthreads();
      // W' = Z0 P^+ (pairs), then V' = W' Sigma
      mm_pair(M, M, N, 1, sPart, [&](int a, int i) { return sZ0[a * N + i]; },
              [&](int i, int b) { return conj_cf(ld4(Pkp[b * N + i])); }, [&](int, int) { return czero(); },
              [&](int a, int b, const cf& v) { sW[a * M + b] = st4(v); });
      __syncthreads();
      mm_pair(M, M, M, 1, sPart, [&](int a, int x) { return ld4(sW[a * M + x]); },
              [&](int x, int b) { return ld4(Sgp[x * M + b]); }, [&](int, int) { return czero(); },
              [&](int a, int b, const cf& v) { sV[a * M + b] = st4(v); });
      __syncthreads();
      // R' = P - Z0 A = P - (i w + mu) Z0 + Z0 H + V' P  (pairs, rounded), M x N
      mm_pair(M, N, N, 1, sPart, [&](int a, int i) { return sZ0[a * N + i]; },
              [&](int i, int c) { return ld4(Hkp[i * N + c]); },
              [&](int a, int c) {
                cf acc = ld4(Pkp[a * N + c]);
                cacc1(acc, zw, sZ0[a * N + c]);
                for (int b = 0; b < M; ++b) cacc(acc, ld4(sV[a * M + b]), ld4(Pkp[b * N + c]));
                return acc;
              },
              [&](int a, int c, const cf& v) { sR[a * N + c] = round_cf(v); });
      __syncthreads();
      // dZ = R' X (FP32)
      mm_f32(M, N, N, [&](int a, int i) { return sR[a * N + i]; }, X,
             [&](int a, int c, float2 v) { sdZ[a * N + c] = v; });
      __syncthreads();
      // B_k = Z Y = Z0 Y0 (pairs of exact FP32 products) + Z0 dY + dZ Y0 (FP32)
      mm_pair(M, M, N, 1, sPart, [&](int a, int i) { return sZ0[a * N + i]; },
              [&](int i, int b) { return sY0[i * M + b]; }, [&](int, int) { return czero(); },
              [&](int a, int b, const cf& v) { sQb[a * M + b] = st4(v); });
      __syncthreads();
      mm_f32(M, M, 2 * N,
             [&](int a, int k) { return k < N ? sZ0[a * N + k] : sdZ[a * N + k - N]; },
             [&](int k, int b) { return k < N ? sdY[k * M + b] : sY0[(k - N) * M + b]; },
             [&](int a, int b, float2 d) {
               cf q = ld4(sQb[a * M + b]);
               add_single(q, d);
               sQb[a * M + b] = st4(q);
             });
      __syncthreads();
      const bool have_gbar = (p.Gbd != nullptr);
      if (have_gbar) {
        const float4* Gb = p.Gbd + si.offSig + (int64_t)n * M * M;
        // Mt = Gbar A_k^+ (pairs)
        mm_pair(M, M, M, 1, sPart, [&](int a, int c) { return ld4(Gb[a * M + c]); },
                [&](int c, int b) { return conj_cf(ld4(sQa[b * M + c])); }, [&](int, int) { return czero(); },
                [&](int a, int b, const cf& v) { sMt[a * M + b] = st4(v); });
        // mu_bar partial: - w_k Re<Gbar, B_k>
        for (int e = tid; e < M * M; e += nthr) {
          const double2 gv = to_d2(ld4(Gb[e])), bv = to_d2(ld4(sQb[e]));
          acc_mu -= wk * fma(gv.x, bv.x, gv.y * bv.y);
        }
        __syncthreads();
      }
      double2* out = p.gq + ((int64_t)(it.g - p.gb0) * p.n_iw + n) * p.mmax * p.mmax;
      const double cb = nbar * 2.0 / beta;
      for (int e = tid; e < M * M; e += nthr) {
        const int a = e / M, b = e - a * M;
        cf acc = czero();
        if (have_gbar)
          for (int c = 0; c < M; ++c) cacc_ca(acc, ld4(sQa[c * M + a]), ld4(sMt[c * M + b]));
        cnorm(acc);
        const double2 v = to_d2(acc);
        const double2 bt = to_d2(ld4(sQb[b * M + a]));
        gq_put(&out[e], q, make_double2(wk * fma(cb, bt.x, v.x), wk * fma(-cb, bt.y, v.y)));
      }
    }
  }
}

template <int RA, int RB, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB) k_point_f32r(const PointParams p) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int s_item;
  __shared__ int s_p[2], s_pq[2], s_pm[2];  // pivot row, its tile index p / TR and p % TR
  __shared__ float2 s_r[2];
  __shared__ double s_red[kMaxWarpsF];
  const LayoutF L = make_layout_f(p.nbmax, p.mmax, p.mode);
  float2* sP = reinterpret_cast<float2*>(smraw + L.oP);
  float2* sS = reinterpret_cast<float2*>(smraw + L.oS);
  float2* sG = reinterpret_cast<float2*>(smraw + L.oG);
  float2* sT = reinterpret_cast<float2*>(smraw + L.oT);
  float2* sB = reinterpret_cast<float2*>(smraw + L.oB);
  float4* sW = reinterpret_cast<float4*>(smraw + L.oW);
  float4* sV = reinterpret_cast<float4*>(smraw + L.oV);
  float2* sY0 = reinterpret_cast<float2*>(smraw + L.oY0);
  float2* sR = reinterpret_cast<float2*>(smraw + L.oR);
  float2* sdY = reinterpret_cast<float2*>(smraw + L.odY);
  float2* sZ0 = reinterpret_cast<float2*>(smraw + L.oZ0);
  float2* sdZ = reinterpret_cast<float2*>(smraw + L.odZ);
  float4* sQa = reinterpret_cast<float4*>(smraw + L.oQa);
  float4* sQb = reinterpret_cast<float4*>(smraw + L.oQb);
  float4* sMt = reinterpret_cast<float4*>(smraw + L.oMt);
  float4* sPart = reinterpret_cast<float4*>(smraw + L.oR);  // partial sums of mm_pair (R and dY regions)
  float2* sD = reinterpret_cast<float2*>(smraw + L.oD);
  double2* sHii = reinterpret_cast<double2*>(smraw + L.oHii);
  int* sPiv = reinterpret_cast<int*>(smraw + L.oPiv);
  int* sIdx = sPiv + p.nbmax;
  int* sRow = sIdx + p.nbmax;
  const int nbp = f32r_nbp(p.nbmax);
  const EpiF eb{sP, sW, sV, sQa, sQb, sMt, sPart, sY0, sR, sdY, sZ0, sdZ};
  float2* bCol = sB;
  float2* bU = sB + 2 * nbp;
  float2* bCx = sB + 4 * nbp;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nthr = blockDim.x;

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
      const int TR = (N + RA - 1) / RA, TC = (N + RB - 1) / RB;
      const int ot = tid - 32;  // warp 0 owns no tile: it runs the pivot lookahead
      const bool owner = ot >= 0 && ot < TR * TC;
      const int tr = owner ? ot / TC : 0, tc = owner ? ot - (ot / TC) * TC : 0;
      const float2* Hk = p.Hs + ki.offH;
      const double2* Hk64 = p.H + ki.offH;
      const float4* Hkp = p.Hd + ki.offH;
      const float4* Pkp = p.Pd + ki.offP;
      const double mu = p.mu[ki.sys];
      const double beta = si.beta;
      const double wk = ki.w;
      double nbar = 0.0;
      if ((p.mode & kAdj) && p.nbar) nbar = p.nbar[ki.sys];
      for (int e = tid; e < M * N; e += nthr) sP[e] = p.Ps[ki.offP + e];
      for (int i = tid; i < N; i += nthr) sHii[i] = Hk64[i * N + i];
      for (int i = tid; i < 2 * nbp; i += nthr) bCol[i] = f2zero();  // zero tails of l
      const double pib = M_PI / beta;

      double acc_tr = 0.0, acc_g2 = 0.0, acc_mu = 0.0;
      for (int n = it.n0; n < it.n1; ++n) {
        const double wn = (2.0 * n + 1.0) * pib;
        __syncthreads();  // previous epilogue done with the shared buffers
        for (int e = tid; e < M * M; e += nthr) sS[e] = p.Ss[si.offSig + (int64_t)n * M * M + e];
        __syncthreads();
        // T = Sigma(i w_n) P_k  (M x N), in the G region
        for (int e = tid; e < M * N; e += nthr) {
          const int a = e / N, j = e - a * N;
          float2 acc = f2zero();
          for (int b = 0; b < M; ++b) fmac(acc, sS[a * M + b], sP[b * N + j]);
          sT[e] = acc;
        }
        for (int i = tid; i < N; i += nthr)
          sD[i] = make_float2(__double2float_rn(mu - sHii[i].x), __double2float_rn(wn - sHii[i].y));
        __syncthreads();
        // A = (i w_n + mu) I - H_k - P_k^+ T in the owners' registers; the diagonal
        // (i w_n + mu - H_ii) comes from sD, formed in FP64 and rounded once
        float2 A[RA][RB];
  #pragma unroll
        for (int a = 0; a < RA; ++a)
  #pragma unroll
          for (int b = 0; b < RB; ++b) {
            const int i = tr + TR * a, c = tc + TC * b;
            float2 v = f2zero();
            if (owner && i < N && c < N) v = (i == c) ? sD[i] : fneg(Hk[i * N + c]);
            A[a][b] = v;
          }
        if (owner) {
          for (int x = 0; x < M; ++x) {
            float2 pv[RA];
  #pragma unroll
            for (int a = 0; a < RA; ++a) {
              const int i = tr + TR * a;
              pv[a] = (i < N) ? fneg(sP[x * N + i]) : f2zero();
            }
  #pragma unroll
            for (int b = 0; b < RB; ++b) {
              const int c = tc + TC * b;
              const float2 tv = (c < N) ? sT[x * N + c] : f2zero();
  #pragma unroll
              for (int a = 0; a < RA; ++a) fmac_ca(A[a][b], pv[a], tv);
            }
          }
        }
        // Gauss-Jordan elimination with partial pivoting, without row interchanges
        // (the exchange or sweep form of the elimination): step j pivots on
        // (p_j, j), p_j the unused row of largest |A[i][j]|, so that afterwards
        // X[i][c] = B[p_i][q_c] with q the inverse permutation of p.  Every step is
        // one uniform rank-1 update of the whole tile,
        //   A[i][c] -= l[i] u[c],  u = A[p][.] / A[p][j] with u[j] = 1/A[p][j],
        //   l[i] = A[i][j] (i != p), l[p] = -1,
        // after the owners of row p and of column j have zeroed them (so that row p
        // becomes u and column j becomes -l u[j]).  Phases per step:
        //  (R) owners of row p publish u and zero the row, owners of column j zero
        //      it, owners of column j+1 publish it (cx);
        //  (U) owners update their tiles; warp 0 applies the same update to cx,
        //      picks p_{j+1} among the unused rows and forms the next l and
        //      1/pivot (one pivot of lookahead).  Two barriers per step.
        if (owner && tc == 0) {
  #pragma unroll
          for (int a = 0; a < RA; ++a) bCx[nbp + tr + TR * a] = A[a][0];
        }
        __syncthreads();
        unsigned used = 0u;  // warp 0: bit t marks row lane + 32 t as a pivot row already
        if (warp == 0) {
          const float2* cx0 = bCx + nbp;
          float2 v[4];
          unsigned best = 0u;
  #pragma unroll
          for (int t = 0; t < 4; ++t) {
            const int i = lane + 32 * t;
            v[t] = (i < N) ? cx0[i] : f2zero();
            if (i < N) best = max(best, pack_key(v[t], i));
          }
          best = __reduce_max_sync(0xffffffffu, best);
          // a zero or non-finite pivot is flagged; the row index stays in range
          const int bi = min(127 - (int)(best & 127u), N - 1);
          if (lane == 0 && ((best >> 7) == 0u || (best & ~127u) >= 0x7f800000u))
            atomicOr(p.status, kFlagSingular);
  #pragma unroll
          for (int t = 0; t < 4; ++t) {
            const int i = lane + 32 * t;
            if (i < N) bCol[i] = (i == bi) ? make_float2(-1.f, 0.f) : v[t];
            if (i == bi) {
              used |= 1u << t;
              s_r[0] = frcp(v[t]);
              s_p[0] = bi;
              s_pq[0] = bi / TR;
              s_pm[0] = bi - (bi / TR) * TR;
              sPiv[0] = bi;
            }
          }
        }
        __syncthreads();
        int jqc = 0, jmc = 0;                                 // j / TC, j % TC
        int nqc = (TC > 1) ? 0 : 1, nmc = (TC > 1) ? 1 : 0;  // (j+1) / TC, (j+1) % TC
        for (int j = 0; j < N; ++j) {
          const int bf = j & 1;
          const float2* col = bCol + bf * nbp;
          float2* urow = bU + bf * nbp;
          float2* cxb = bCx + bf * nbp;
          const int prq = s_pq[bf], prm = s_pm[bf];
          const float2 r = s_r[bf];
          const int jn = j + 1;
          if (owner) {
            if (tr == prm) {
  #pragma unroll
              for (int a = 0; a < RA; ++a)
                if (a == prq) {
  #pragma unroll
                  for (int b = 0; b < RB; ++b) {
                    const int c = tc + TC * b;
                    urow[c] = (c == j) ? r : fmul(A[a][b], r);
                    A[a][b] = f2zero();
                  }
                }
            }
            if (tc == jmc) {
  #pragma unroll
              for (int b = 0; b < RB; ++b)
                if (b == jqc) {
  #pragma unroll
                  for (int a = 0; a < RA; ++a) A[a][b] = f2zero();
                }
            }
            if (jn < N && tc == nmc) {
  #pragma unroll
              for (int b = 0; b < RB; ++b)
                if (b == nqc) {
  #pragma unroll
                  for (int a = 0; a < RA; ++a) cxb[tr + TR * a] = A[a][b];
                }
            }
          }
          __syncthreads();
          if (owner) {
            float2 lv[RA];
  #pragma unroll
            for (int a = 0; a < RA; ++a) lv[a] = col[tr + TR * a];
  #pragma unroll
            for (int b = 0; b < RB; ++b) {
              const float2 u = urow[tc + TC * b];
  #pragma unroll
              for (int a = 0; a < RA; ++a) fsub_prod(A[a][b], lv[a], u);
            }
          } else if (warp == 0 && jn < N) {
            float2* ncol = bCol + (bf ^ 1) * nbp;
            const float2 u = urow[jn];
            float2 v[4];
            unsigned best = 0u;
  #pragma unroll
            for (int t = 0; t < 4; ++t) {
              const int i = lane + 32 * t;
              v[t] = f2zero();
              if (i < N) {
                v[t] = cxb[i];
                fsub_prod(v[t], col[i], u);
                if (!((used >> t) & 1u)) best = max(best, pack_key(v[t], i));
              }
            }
            best = __reduce_max_sync(0xffffffffu, best);
            const int bi = min(127 - (int)(best & 127u), N - 1);
            if (lane == 0 && ((best >> 7) == 0u || (best & ~127u) >= 0x7f800000u))
              atomicOr(p.status, kFlagSingular);
  #pragma unroll
            for (int t = 0; t < 4; ++t) {
              const int i = lane + 32 * t;
              if (i < N) ncol[i] = (i == bi) ? make_float2(-1.f, 0.f) : v[t];
              if (i == bi) {
                used |= 1u << t;
                s_r[bf ^ 1] = frcp(v[t]);
                s_p[bf ^ 1] = bi;
                s_pq[bf ^ 1] = bi / TR;
                s_pm[bf ^ 1] = bi - (bi / TR) * TR;
                sPiv[jn] = bi;
              }
            }
          }
          __syncthreads();
          if (++jmc == TC) { jmc = 0; ++jqc; }
          if (++nmc == TC) { nmc = 0; ++nqc; }
        }
        // B to shared memory; X[i][c] = B[p_i][q_c]: sPiv = p, sIdx = q = p^{-1}
        if (owner) {
  #pragma unroll
          for (int a = 0; a < RA; ++a)
  #pragma unroll
            for (int b = 0; b < RB; ++b) {
              const int i = tr + TR * a, c = tc + TC * b;
              if (i < N && c < N) sG[i * ld + c] = A[a][b];
            }
        }
        for (int j = tid; j < N; j += nthr) sIdx[sPiv[j]] = j;
        __syncthreads();
        for (int i = tid; i < N; i += nthr) sRow[i] = sPiv[i] * ld;
        __syncthreads();

        if (p.mode & kOcc) {
          for (int i = tid; i < N; i += nthr) acc_tr += (double)sG[sRow[i] + sIdx[i]].x;
          float g2 = 0.f;
          for (int e = tid; e < N * N; e += nthr) {
            const int i = e / N, c = e - i * N;
            const float2 g1 = sG[sRow[i] + sIdx[c]], gt = sG[sRow[c] + sIdx[i]];
            g2 = __fmaf_rn(g1.x, gt.x, __fmaf_rn(-g1.y, gt.y, g2));
          }
          acc_g2 += (double)g2;
        }
        f32r_epilogues(p, eb, it, ki, si, q, N, M, n, wn, mu, beta, wk, nbar, Hkp, Pkp, sG, sRow, sIdx,
                       acc_mu);
      }
      if (p.mode & kOcc) {
        const double tr_ = block_sum_f(acc_tr, s_red);
        const double g2 = block_sum_f(acc_g2, s_red);
        if (tid == 0) {
          double* o = p.occ_part + ((int64_t)kk * p.n_chunks + it.chunk) * 2;
          o[0] = tr_;
          o[1] = g2;
        }
      }
      if (p.mode & kAdj) {
        const double mb = block_sum_f(acc_mu, s_red);
        if (tid == 0) p.mubar_part[(int64_t)kk * p.n_chunks + it.chunk] = mb;
      }
      __syncthreads();
    }
  }
}

// Tile shapes: (RA, RB), the thread bound of the instantiation (owners plus the
// pivot warp), the minimum resident CTAs it is compiled for, and the largest
// window it is meant for (TR = ceil(N / RA), TC = ceil(N / RB), TR TC <= MAXT - 32).
struct ShapeF {
  int ra, rb, maxt, minb, nmax;
};
constexpr ShapeF kShapesF[] = {
    {2, 2, 96, 4, 16},   {2, 5, 192, 3, 40},  {4, 5, 128, 4, 40},  {4, 4, 288, 2, 64},
    {4, 8, 160, 3, 64},  {6, 8, 224, 2, 96},  {4, 8, 352, 1, 96},  {4, 8, 544, 1, 128},
    {8, 8, 288, 1, 128}, {4, 4, 640, 1, 96},  {4, 6, 736, 1, 128},
};
constexpr int kNumShapesF = (int)(sizeof(kShapesF) / sizeof(kShapesF[0]));

template <int RA, int RB, int MAXT, int MINB>
cudaError_t launch_f(const PointParams& p, int grid, int threads, size_t smem, cudaStream_t s) {
  if (threads > MAXT) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_point_f32r<RA, RB, MAXT, MINB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_point_f32r<RA, RB, MAXT, MINB><<<grid, threads, smem, s>>>(p);
  return cudaGetLastError();
}

template <int RA, int RB, int MAXT, int MINB>
int bps_f(int threads, size_t smem) {
  int nb = 0;
  if (cudaFuncSetAttribute(k_point_f32r<RA, RB, MAXT, MINB>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_point_f32r<RA, RB, MAXT, MINB>, threads,
                                                    smem) != cudaSuccess)
    return 0;
  return nb;
}

#define GF_F32R_SHAPES(X) \
  X(0, 2, 2, 96, 4)       \
  X(1, 2, 5, 192, 3)      \
  X(2, 4, 5, 128, 4)      \
  X(3, 4, 4, 288, 2)      \
  X(4, 4, 8, 160, 3)      \
  X(5, 6, 8, 224, 2)      \
  X(6, 4, 8, 352, 1)      \
  X(7, 4, 8, 544, 1)      \
  X(8, 8, 8, 288, 1)      \
  X(9, 4, 4, 640, 1)      \
  X(10, 4, 6, 736, 1)

}  // namespace

int f32r_num_shapes() { return kNumShapesF; }

int f32r_tile(int shape, int which) {
  if (shape < 0 || shape >= kNumShapesF) return 0;
  return which == 0 ? kShapesF[shape].ra : kShapesF[shape].rb;
}

// A shape serves a window of nbmax bands when its owner grid fits its thread
// bound and nbmax is within the window class it was tuned for.
bool f32r_shape_fits(int shape, int nbmax) {
  if (shape < 0 || shape >= kNumShapesF) return false;
  const ShapeF sh = kShapesF[shape];
  if (nbmax > sh.nmax) return false;
  return ((nbmax + sh.ra - 1) / sh.ra) * ((nbmax + sh.rb - 1) / sh.rb) <= sh.maxt - 32;
}

int f32r_threads(int shape, int nbmax) {
  const ShapeF sh = kShapesF[shape];
  const int t = ((nbmax + sh.ra - 1) / sh.ra) * ((nbmax + sh.rb - 1) / sh.rb);
  return 32 + ((t + 31) / 32) * 32;  // owners plus the pivot warp
}

int f32r_nmax(int shape) { return (shape >= 0 && shape < kNumShapesF) ? kShapesF[shape].nmax : 0; }

size_t point_f32r_smem(int nbmax, int mmax, int mode) { return make_layout_f(nbmax, mmax, mode).bytes; }

int point_f32r_blocks_per_sm(int shape, int threads, size_t smem) {
  switch (shape) {
#define X(i, a, b, t, m) \
  case i:                \
    return bps_f<a, b, t, m>(threads, smem);
    GF_F32R_SHAPES(X)
#undef X
  }
  return 0;
}

cudaError_t launch_point_f32r(int shape, const PointParams& p, int grid, int threads, size_t smem,
                              cudaStream_t s) {
  switch (shape) {
#define X(i, a, b, t, m) \
  case i:                \
    return launch_f<a, b, t, m>(p, grid, threads, smem, s);
    GF_F32R_SHAPES(X)
#undef X
  }
  return cudaErrorInvalidValue;
}


// Shared memory of k_point_f32w (bytes): the CTA's P and H_ii of the k-point and the
// epilogue buffers (as in LayoutF; R and dY contiguous for the pair partial sums), then
// per warp Sigma, T = Sigma P (then the warp's inverse), the diagonal, the pivot-row
// buffer and the pivot tables.
struct LayoutFW {
  size_t oP, oHii, oW, oV, oY0, oR, odY, oZ0, odZ, oQa, oQb, oMt, warp0, wstride, wS, wX, wD, wBuf, wPiv, bytes;
};

__host__ __device__ inline LayoutFW make_layout_fw(int nbmax, int mmax, int mode, int nmax, int nwarps) {
  LayoutFW L;
  const size_t ld = (size_t)(nbmax | 1);
  const size_t mn = (size_t)mmax * nbmax, mm = (size_t)mmax * mmax;
  const bool refine = (mode & (kGloc | kAdj)) != 0;
  const bool adj = (mode & kAdj) != 0;
  size_t o = 0;
  auto take = [&o](size_t bytes) {  // 16-byte aligned region
    o = (o + 15) & ~(size_t)15;
    const size_t at = o;
    o += bytes;
    return at;
  };
  L.oP = take(8 * mn);
  L.oHii = take(16 * (size_t)nbmax);
  L.oW = take(refine ? 16 * mm : 0);
  L.oV = take(refine ? 16 * mm : 0);
  L.oY0 = take(refine ? 8 * mn : 0);
  L.oR = take(refine ? 8 * mn : 0);
  L.odY = o; o += refine ? 8 * mn : 0;
  L.oZ0 = take(adj ? 8 * mn : 0);
  L.odZ = take(adj ? 8 * mn : 0);
  L.oQa = take(adj ? 16 * mm : 0);
  L.oQb = take(adj ? 16 * mm : 0);
  L.oMt = take(adj ? 16 * mm : 0);
  L.warp0 = take(0);
  size_t g = 0;
  auto wtake = [&g](size_t bytes) {
    g = (g + 15) & ~(size_t)15;
    const size_t at = g;
    g += bytes;
    return at;
  };
  size_t x = mn;
  if (x < (size_t)nbmax * ld) x = (size_t)nbmax * ld;
  L.wS = wtake(8 * mm);
  L.wX = wtake(8 * x);
  L.wD = wtake(8 * (size_t)nbmax);
  L.wBuf = wtake(8 * (size_t)nmax);
  L.wPiv = wtake(3 * sizeof(int) * (size_t)nmax);
  L.wstride = (g + 15) & ~(size_t)15;
  L.bytes = L.warp0 + (size_t)nwarps * L.wstride;
  return L;
}

namespace {

constexpr int kF32wWarps = 4;  // warps per CTA: frequencies inverted together

// Fused passes (kRho, kGloc, kAdj, with or without kOcc) for windows up to 40 bands.
// Each warp inverts one frequency of the item with warp_invert (one warp per matrix,
// the matrix in registers; kOcc traces taken by the warp from its inverse), then the
// whole CTA runs the refined-projection epilogues of the W inverses in frequency order.
template <int NMAX, bool SPLIT, int W>
__global__ void __launch_bounds__(32 * W, 2) k_point_f32w(const PointParams p) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int s_item;
  __shared__ double s_red[W];
  const LayoutFW L = make_layout_fw(p.nbmax, p.mmax, p.mode, NMAX, W);
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  float2* sP = reinterpret_cast<float2*>(smraw + L.oP);
  double2* sHii = reinterpret_cast<double2*>(smraw + L.oHii);
  const EpiF eb{sP,
                reinterpret_cast<float4*>(smraw + L.oW),
                reinterpret_cast<float4*>(smraw + L.oV),
                reinterpret_cast<float4*>(smraw + L.oQa),
                reinterpret_cast<float4*>(smraw + L.oQb),
                reinterpret_cast<float4*>(smraw + L.oMt),
                reinterpret_cast<float4*>(smraw + L.oR),
                reinterpret_cast<float2*>(smraw + L.oY0),
                reinterpret_cast<float2*>(smraw + L.oR),
                reinterpret_cast<float2*>(smraw + L.odY),
                reinterpret_cast<float2*>(smraw + L.oZ0),
                reinterpret_cast<float2*>(smraw + L.odZ)};
  auto warp_region = [&](int w) { return smraw + L.warp0 + (size_t)w * L.wstride; };
  auto bufs_of = [&](int w) {
    unsigned char* wb = warp_region(w);
    int* piv = reinterpret_cast<int*>(wb + L.wPiv);
    return wgj::WarpBufs{reinterpret_cast<float2*>(wb + L.wX), reinterpret_cast<float2*>(wb + L.wBuf), piv,
                         piv + NMAX, piv + 2 * NMAX};
  };
  float2* sS = reinterpret_cast<float2*>(warp_region(wp) + L.wS);
  float2* sD = reinterpret_cast<float2*>(warp_region(wp) + L.wD);
  const wgj::WarpBufs mine = bufs_of(wp);

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
      const int N = ki.nb, M = si.m;
      const float2* Hk = p.Hs + ki.offH;
      const double2* Hk64 = p.H + ki.offH;
      const float4* Hkp = p.Hd + ki.offH;
      const float4* Pkp = p.Pd + ki.offP;
      const double mu = p.mu[ki.sys];
      const double beta = si.beta;
      const double wk = ki.w;
      double nbar = 0.0;
      if ((p.mode & kAdj) && p.nbar) nbar = p.nbar[ki.sys];
      for (int e = tid; e < M * N; e += 32 * W) sP[e] = p.Ps[ki.offP + e];
      for (int i = tid; i < N; i += 32 * W) sHii[i] = Hk64[i * N + i];
      __syncthreads();
      const double pib = M_PI / beta;
      double acc_tr = 0.0, acc_g2 = 0.0, acc_mu = 0.0;
      for (int nb = it.n0; nb < it.n1; nb += W) {
        // every warp inverts one frequency
        const int n = nb + wp;
        if (n < it.n1) {
          const double wn = (2.0 * n + 1.0) * pib;
          wgj::warp_point_inputs(p.Ss + si.offSig + (int64_t)n * M * M, sHii, sP, mu, wn, N, M, lane, sS, sD,
                                 mine.sX);
          wgj::warp_invert<NMAX, SPLIT>(Hk, sD, sP, mine, N, M, lane, p.status);
          if (p.mode & kOcc) {
            const float2* sX = mine.sX;
            for (int x = lane; x < N; x += 32) acc_tr += (double)sX[mine.sRow[x] + mine.sIdx[x]].x;
            float g2 = 0.f;
            for (int e = lane; e < N * N; e += 32) {
              const int i = e / N, c = e - i * N;
              const float2 g1 = sX[mine.sRow[i] + mine.sIdx[c]], g3 = sX[mine.sRow[c] + mine.sIdx[i]];
              g2 = __fmaf_rn(g1.x, g3.x, __fmaf_rn(-g1.y, g3.y, g2));
            }
            acc_g2 += (double)g2;
          }
        }
        __syncthreads();  // the inverses of the batch are visible to the CTA
        // the CTA's epilogues, one frequency after the other
        const int nw = min(W, it.n1 - nb);
        for (int w = 0; w < nw; ++w) {
          const int nn = nb + w;
          const wgj::WarpBufs bw = bufs_of(w);
          f32r_epilogues(p, eb, it, ki, si, q, N, M, nn, (2.0 * nn + 1.0) * pib, mu, beta, wk, nbar, Hkp, Pkp,
                         bw.sX, bw.sRow, bw.sIdx, acc_mu);
          __syncthreads();  // epilogue buffers and the warp regions free again
        }
      }
      if (p.mode & kOcc) {
        const double tr_ = block_sum_f(acc_tr, s_red);
        const double g2 = block_sum_f(acc_g2, s_red);
        if (tid == 0) {
          double* o = p.occ_part + ((int64_t)kk * p.n_chunks + it.chunk) * 2;
          o[0] = tr_;
          o[1] = g2;
        }
      }
      if (p.mode & kAdj) {
        const double mb = block_sum_f(acc_mu, s_red);
        if (tid == 0) p.mubar_part[(int64_t)kk * p.n_chunks + it.chunk] = mb;
      }
      __syncthreads();
    }
  }
}

template <int NMAX, bool SPLIT>
cudaError_t set_attrs_fw(size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(k_point_f32w<NMAX, SPLIT, kF32wWarps>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_point_f32w<NMAX, SPLIT, kF32wWarps>, cudaFuncAttributePreferredSharedMemoryCarveout,
                              (int)cudaSharedmemCarveoutMaxShared);
}

template <int NMAX, bool SPLIT>
cudaError_t launch_fw(const PointParams& p, int grid, size_t smem, cudaStream_t s) {
  const cudaError_t e = set_attrs_fw<NMAX, SPLIT>(smem);
  if (e != cudaSuccess) return e;
  k_point_f32w<NMAX, SPLIT, kF32wWarps><<<grid, 32 * kF32wWarps, smem, s>>>(p);
  return cudaGetLastError();
}

template <int NMAX, bool SPLIT>
int bps_fw(size_t smem) {
  int nb = 0;
  if (set_attrs_fw<NMAX, SPLIT>(smem) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_point_f32w<NMAX, SPLIT, kF32wWarps>, 32 * kF32wWarps,
                                                    smem) != cudaSuccess)
    return 0;
  return nb;
}

}  // namespace

// Largest window of the instantiation that serves nbmax, or 0 (the one-warp inverse
// holds windows up to 40 bands).
int f32w_nmax(int nbmax) { return nbmax <= 16 ? 16 : (nbmax <= 32 ? 32 : (nbmax <= 40 ? 40 : 0)); }

int f32w_threads() { return 32 * kF32wWarps; }

size_t point_f32w_smem(int nbmax, int mmax, int mode) {
  return make_layout_fw(nbmax, mmax, mode, f32w_nmax(nbmax), kF32wWarps).bytes;
}

int point_f32w_blocks_per_sm(int nbmax, size_t smem) {
  switch (f32w_nmax(nbmax)) {
    case 16: return bps_fw<16, false>(smem);
    case 32: return bps_fw<32, false>(smem);
    case 40: return bps_fw<40, true>(smem);
    default: return 0;
  }
}

cudaError_t launch_point_f32w(int nbmax, const PointParams& p, int grid, size_t smem, cudaStream_t s) {
  switch (f32w_nmax(nbmax)) {
    case 16: return launch_fw<16, false>(p, grid, smem, s);
    case 32: return launch_fw<32, false>(p, grid, smem, s);
    case 40: return launch_fw<40, true>(p, grid, smem, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace gf

namespace gf {

namespace {
__global__ void k_round_f32(const double2* __restrict__ in, float2* __restrict__ out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = make_float2(__double2float_rn(in[i].x), __double2float_rn(in[i].y));
}
}  // namespace

cudaError_t launch_round_f32(const double2* in, float2* out, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_round_f32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, out, n);
  return cudaGetLastError();
}

}  // namespace gf

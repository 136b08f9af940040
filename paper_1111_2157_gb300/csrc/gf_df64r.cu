// Register-resident FP32-pair kernel of the lattice Green's function path (sm_103a).
//
// Same arithmetic as gf_df64.cu (every entry an unevaluated sum hi + lo of two
// FP32 numbers, error-free transformations on the FP32 pipes), with the matrix
// held in registers during the Gauss-Jordan inverse instead of shared memory.
// The CTA is a TR x TC thread grid; thread (tr, tc) owns the RA x RB entries
// (tr + TR a, tc + TC b).  A pivot step then reads, per thread, RA multipliers
// and RB pivot-row entries from shared memory (broadcast) for RA * RB updates,
// where the shared-memory version moved 64 bytes per update.  The embedding
// A = (i w + mu) - H - P^+ (Sigma P) is formed directly in the owners'
// registers as RA * RB independent accumulators.  After the inverse the tile is
// written once to shared memory and the epilogues (traces, rho, G_loc, adjoint)
// run on that copy exactly as in the shared-memory kernels.
#include <math.h>
#include <stdint.h>

#include "gf_complex.cuh"
#include "gf_internal.cuh"

namespace gf {

namespace {

using namespace cx;


constexpr int kMaxWarps = 16;

// Deterministic block sum for any blockDim that is a multiple of 32 (<= 512).
__device__ __forceinline__ double block_sum_any(double v, double* red) {
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

// Shared memory (16-byte elements): P_k | T (Sigma P, then Y) | Sigma / Gbar |
// G copy (N x ld) | col x2 | urow x2 | rowj x2 | next column x2 | Z | A_k | B_k,
// then piv, idx.
struct LayoutR {
  int offP, offT, offS, offG, offCol, offU, offRj, offCx, offZ, offQa, offQb, n16;
  size_t bytes;
};
__host__ __device__ inline LayoutR make_layout_r(int nbmax, int mmax, int mode) {
  LayoutR L;
  const int ld = nbmax | 1;
  int o = 0;
  L.offP = o; o += mmax * nbmax;
  L.offT = o; o += imax(mmax * nbmax, mmax * mmax);
  L.offS = o; o += mmax * mmax;
  L.offG = o; o += nbmax * ld;
  L.offCol = o; o += 2 * nbmax;
  L.offU = o; o += 2 * nbmax;
  L.offRj = o; o += 2 * nbmax;
  L.offCx = o; o += 2 * nbmax;
  L.offZ = o; o += (mode & kAdj) ? mmax * nbmax : 0;
  L.offQa = o; o += (mode & kAdj) ? mmax * mmax : 0;
  L.offQb = o; o += (mode & kAdj) ? mmax * mmax : 0;
  L.n16 = o;
  L.bytes = (size_t)o * 16 + 2 * (size_t)nbmax * sizeof(int);
  return L;
}

template <int RA, int RB, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB) k_point_df64r(const PointParams p) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float4* sm = reinterpret_cast<float4*>(smraw);
  __shared__ int s_item;
  __shared__ int s_p[2], s_pq[2], s_pm[2];  // pivot row, its tile row index p / TR and p % TR
  __shared__ float4 s_r[2];
  __shared__ double s_red[kMaxWarps];
  const LayoutR L = make_layout_r(p.nbmax, p.mmax, p.mode);
  float4* sP = sm + L.offP;
  float4* sT = sm + L.offT;
  float4* sS = sm + L.offS;
  float4* sG = sm + L.offG;
  float4* sZ = sm + L.offZ;
  float4* sQa = sm + L.offQa;
  float4* sQb = sm + L.offQb;
  int* sPiv = reinterpret_cast<int*>(sm + L.n16);
  int* sIdx = sPiv + p.nbmax;
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
      // thread grid of this k-point's window
      const int TR = (N + RA - 1) / RA, TC = (N + RB - 1) / RB;
      const int ot = tid - 32;  // warp 0 owns no tile: it runs the pivot lookahead
      const bool owner = ot >= 0 && ot < TR * TC;
      const int tr = owner ? ot / TC : 0, tc = owner ? ot - (ot / TC) * TC : 0;
      const float4* Hk = p.Hd + ki.offH;
      const float4* Pg = p.Pd + ki.offP;
      const double mu = p.mu[ki.sys];
      const double beta = si.beta;
      const double wk = ki.w;
      double nbar = 0.0;
      if ((p.mode & kAdj) && p.nbar) nbar = p.nbar[ki.sys];
      float mu_h, mu_l;
      split(mu, mu_h, mu_l);
      for (int e = tid; e < M * N; e += nthr) sP[e] = Pg[e];

      double acc_tr = 0.0, acc_mu = 0.0;
      float g2h = 0.f, g2l = 0.f;
      for (int n = it.n0; n < it.n1; ++n) {
        __syncthreads();
        for (int e = tid; e < M * M; e += nthr) sS[e] = p.Sd[si.offSig + (int64_t)n * M * M + e];
        __syncthreads();
        // T = Sigma(i w_n) P_k
        for (int e = tid; e < M * N; e += nthr) {
          const int a = e / N, j = e - a * N;
          cf acc = czero();
          for (int b = 0; b < M; ++b) cacc(acc, ld4(sS[a * M + b]), ld4(sP[b * N + j]));
          cnorm(acc);
          sT[e] = st4(acc);
        }
        __syncthreads();
        // A = (i w_n + mu) I - H_k - P_k^+ T, formed in the owners' registers
        cf A[RA][RB];
        {
          float wn_h, wn_l;
          split((2.0 * n + 1.0) * M_PI / beta, wn_h, wn_l);
  #pragma unroll
          for (int a = 0; a < RA; ++a)
  #pragma unroll
            for (int b = 0; b < RB; ++b) {
              const int i = tr + TR * a, c = tc + TC * b;
              A[a][b] = (owner && i < N && c < N) ? cneg(ld4(Hk[i * N + c])) : czero();
              if (owner && i == c && i < N) {
                float s, t;
                two_sum(A[a][b].rh, mu_h, s, t);
                A[a][b].rh = s;
                A[a][b].rl = __fadd_rn(A[a][b].rl, __fadd_rn(t, mu_l));
                two_sum(A[a][b].ih, wn_h, s, t);
                A[a][b].ih = s;
                A[a][b].il = __fadd_rn(A[a][b].il, __fadd_rn(t, wn_l));
              }
            }
          if (owner) {
            for (int x = 0; x < M; ++x) {
              cf pv[RA];
  #pragma unroll
              for (int a = 0; a < RA; ++a) {
                const int i = tr + TR * a;
                pv[a] = (i < N) ? cneg(ld4(sP[x * N + i])) : czero();
              }
  #pragma unroll
              for (int b = 0; b < RB; ++b) {
                const int c = tc + TC * b;
                const cf tv = (c < N) ? ld4(sT[x * N + c]) : czero();
  #pragma unroll
                for (int a = 0; a < RA; ++a) cacc_ca(A[a][b], pv[a], tv);
              }
            }
  #pragma unroll
            for (int a = 0; a < RA; ++a)
  #pragma unroll
              for (int b = 0; b < RB; ++b) cnorm(A[a][b]);
          }
        }
        // Gauss-Jordan with partial pivoting on the register tiles, one pivot of
        // lookahead.  Before step j the multipliers l = col (l[j] = 0,
        // l[p] = A[j][j], l[i] = A[i][j]), the pivot row p and r = 1/pivot are known.
        //  (R) owners of row p publish urow = r A[p][.] (urow[j] = r), owners of
        //      row j publish the old row j (rowj), owners of column j+1 publish
        //      their column j+1 (cnx);
        //  (U) owners zero column j, replace row j by urow and row p by rowj, and
        //      update every owned entry a -= l[i] urow[c]; meanwhile warp 0 applies
        //      the same operations to cnx, searches the new column j+1 for the
        //      next pivot, forms its reciprocal and the next multipliers.
        // Two barriers per pivot; the search and the reciprocal overlap the update.
        if (owner && tc == 0) {
  #pragma unroll
          for (int a = 0; a < RA; ++a) {
            const int i = tr + TR * a;
            if (i < N) sm[L.offCx + p.nbmax + i] = st4(A[a][0]);
          }
        }
        __syncthreads();
        if (warp == 0) {
          // pivot of column 0 from the published column (no transformation yet)
          const float4* cx = sm + L.offCx + p.nbmax;
          float4* col = sm + L.offCol;
          unsigned best = 0u;
          int bi = 0x7fffffff;
          for (int i = lane; i < N; i += 32) {
            const unsigned key = pivot_key_f(cx[i]);
            if (bi == 0x7fffffff || key > best) { best = key; bi = i; }
          }
          for (int off = 16; off; off >>= 1) {
            const unsigned ob = __shfl_xor_sync(0xffffffffu, best, off);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
          }
          for (int i = lane; i < N; i += 32) col[i] = (i == 0) ? make_float4(0.f, 0.f, 0.f, 0.f)
                                                              : ((i == bi) ? cx[0] : cx[i]);
          if (lane == 0) {
            if (best == 0u || best >= 0x7f800000u) atomicOr(p.status, kFlagSingular);
            s_p[0] = bi;
            s_pq[0] = bi / TR;
            s_pm[0] = bi - (bi / TR) * TR;
            s_r[0] = st4(crcp_df(ld4(cx[bi])));
            sPiv[0] = bi;
          }
        }
        __syncthreads();
        int jqr = 0, jmr = 0, jqc = 0, jmc = 0;  // j / TR, j % TR, j / TC, j % TC
        int nqc = (TC > 1) ? 0 : 1, nmc = (TC > 1) ? 1 : 0;  // (j+1) / TC, (j+1) % TC
        for (int j = 0; j < N; ++j) {
          const int bf = j & 1;
          float4* col = sm + L.offCol + bf * p.nbmax;
          float4* urow = sm + L.offU + bf * p.nbmax;
          float4* rowj = sm + L.offRj + bf * p.nbmax;
          float4* cx = sm + L.offCx + bf * p.nbmax;
          const int pr = s_p[bf], prq = s_pq[bf], prm = s_pm[bf];
          const cf r = ld4(s_r[bf]);
          const int jn = j + 1;
          if (owner) {
            if (tr == prm) {
  #pragma unroll
              for (int a = 0; a < RA; ++a)
                if (a == prq)
  #pragma unroll
                  for (int b = 0; b < RB; ++b) {
                    const int c = tc + TC * b;
                    if (c < N) {
                      cf u = r;
                      if (c != j) {
                        u = czero();
                        cacc(u, A[a][b], r);
                        cnorm(u);
                      }
                      urow[c] = st4(u);
                    }
                  }
            }
            if (tr == jmr) {
  #pragma unroll
              for (int a = 0; a < RA; ++a)
                if (a == jqr)
  #pragma unroll
                  for (int b = 0; b < RB; ++b) {
                    const int c = tc + TC * b;
                    if (c < N) rowj[c] = st4(A[a][b]);
                  }
            }
            if (jn < N && tc == nmc) {
  #pragma unroll
              for (int a = 0; a < RA; ++a)
  #pragma unroll
                for (int b = 0; b < RB; ++b)
                  if (b == nqc) {
                    const int i = tr + TR * a;
                    if (i < N) cx[i] = st4(A[a][b]);
                  }
            }
          }
          __syncthreads();
          if (owner) {
            const bool own_j = (tr == jmr), own_p = (pr != j && tr == prm);
            if (own_j || own_p) {
  #pragma unroll
              for (int a = 0; a < RA; ++a)
  #pragma unroll
                for (int b = 0; b < RB; ++b) {
                  const int c = tc + TC * b;
                  if (c < N) {
                    if (own_p && a == prq && c != j) A[a][b] = ld4(rowj[c]);
                  }
                }
            }
            if (tc == jmc) {
  #pragma unroll
              for (int a = 0; a < RA; ++a)
  #pragma unroll
                for (int b = 0; b < RB; ++b)
                  if (b == jqc) A[a][b] = czero();
            }
            if (own_j) {
  #pragma unroll
              for (int a = 0; a < RA; ++a)
                if (a == jqr)
  #pragma unroll
                  for (int b = 0; b < RB; ++b) {
                    const int c = tc + TC * b;
                    if (c < N) A[a][b] = ld4(urow[c]);
                  }
            }
            cf lv[RA];
  #pragma unroll
            for (int a = 0; a < RA; ++a) {
              const int i = tr + TR * a;
              lv[a] = (i < N) ? ld4(col[i]) : czero();
            }
  #pragma unroll
            for (int b = 0; b < RB; ++b) {
              const int c = tc + TC * b;
              const cf u = (c < N) ? ld4(urow[c]) : czero();
  #pragma unroll
              for (int a = 0; a < RA; ++a) csub_prod(A[a][b], lv[a], u);
            }
          } else if (warp == 0 && jn < N) {
            // lookahead: column j+1 after step j, exactly as its owners compute it
            float4* ncol = sm + L.offCol + (bf ^ 1) * p.nbmax;
            const cf u = ld4(urow[jn]);
            unsigned best = 0u;
            int bi = 0x7fffffff;
            for (int i = lane; i < N; i += 32) {
              cf v;
              if (i == j) v = ld4(urow[jn]);
              else if (i == pr) v = ld4(rowj[jn]);
              else v = ld4(cx[i]);
              csub_prod(v, ld4(col[i]), u);
              cx[i] = st4(v);
              if (i >= jn) {
                const unsigned key = pivot_key_f(cx[i]);
                if (bi == 0x7fffffff || key > best) { best = key; bi = i; }
              }
            }
            for (int off = 16; off; off >>= 1) {
              const unsigned ob = __shfl_xor_sync(0xffffffffu, best, off);
              const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
              if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            __syncwarp();
            for (int i = lane; i < N; i += 32)
              ncol[i] = (i == jn) ? make_float4(0.f, 0.f, 0.f, 0.f) : ((i == bi) ? cx[jn] : cx[i]);
            if (lane == 0) {
              if (best == 0u || best >= 0x7f800000u) atomicOr(p.status, kFlagSingular);
              s_p[bf ^ 1] = bi;
              s_pq[bf ^ 1] = bi / TR;
              s_pm[bf ^ 1] = bi - (bi / TR) * TR;
              s_r[bf ^ 1] = st4(crcp_df(ld4(cx[bi])));
              sPiv[jn] = bi;
            }
          }
          __syncthreads();
          if (++jmr == TR) { jmr = 0; ++jqr; }
          if (++jmc == TC) { jmc = 0; ++jqc; }
          if (++nmc == TC) { nmc = 0; ++nqc; }
        }
        // inverse (columns permuted by idx) to shared memory for the epilogues
        if (owner) {
  #pragma unroll
          for (int a = 0; a < RA; ++a)
  #pragma unroll
            for (int b = 0; b < RB; ++b) {
              const int i = tr + TR * a, c = tc + TC * b;
              if (i < N && c < N) sG[i * ld + c] = st4(A[a][b]);
            }
        }
        if (tid == 0) {
          for (int c = 0; c < N; ++c) sIdx[c] = c;
          for (int j = N - 1; j >= 0; --j) {
            const int pp = sPiv[j];
            if (pp != j) { const int t = sIdx[j]; sIdx[j] = sIdx[pp]; sIdx[pp] = t; }
          }
        }
        __syncthreads();

        if (p.mode & kOcc) {
          for (int i = tid; i < N; i += nthr) {
            const float4 gv = sG[i * ld + sIdx[i]];
            acc_tr += (double)gv.x + (double)gv.y;
          }
          for (int e = tid; e < N * N; e += nthr) {
            const int i = e / N, c = e - i * N;
            const float4 g1 = sG[i * ld + sIdx[c]], g2 = sG[c * ld + sIdx[i]];
            acc_prod(g1.x, g1.y, g2.x, g2.y, g2h, g2l);
            acc_prod(-g1.z, -g1.w, g2.z, g2.w, g2h, g2l);
          }
          renorm(g2h, g2l);
        }
        if (p.mode & kRho) {
          double2* S = p.rho_part + (int64_t)it.chunk * p.rho_chunk_stride + ki.offH;
          const bool first = (n == it.n0);
          for (int e = tid; e < N * N; e += nthr) {
            const int i = e / N, c = e - i * N;
            const double2 gv = to_d2(ld4(sG[i * ld + sIdx[c]]));
            if (first) {
              S[e] = gv;
            } else {
              double2 s = S[e];
              s.x += gv.x;
              s.y += gv.y;
              S[e] = s;
            }
          }
        }
        if (p.mode & (kGloc | kAdj)) {
          for (int e = tid; e < N * M; e += nthr) {
            const int i = e / M, b = e - i * M;
            cf acc = czero();
            for (int c = 0; c < N; ++c) {
              cacc_cb(acc, ld4(sG[i * ld + sIdx[c]]), ld4(sP[b * N + c]));
              if ((c & 15) == 15) cnorm(acc);
            }
            cnorm(acc);
            sT[e] = st4(acc);
          }
          if (p.mode & kAdj) {
            for (int e = tid; e < M * N; e += nthr) {
              const int a = e / N, c = e - a * N;
              const int colx = sIdx[c];
              cf acc = czero();
              for (int i = 0; i < N; ++i) {
                cacc(acc, ld4(sP[a * N + i]), ld4(sG[i * ld + colx]));
                if ((i & 15) == 15) cnorm(acc);
              }
              cnorm(acc);
              sZ[e] = st4(acc);
            }
          }
          __syncthreads();
          if (p.mode & kGloc) {
            double2* out = p.gq + ((int64_t)(it.g - p.gb0) * p.n_iw + n) * p.mmax * p.mmax;
            for (int e = tid; e < M * M; e += nthr) {
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
            for (int e = tid; e < M * M; e += nthr) {
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
              for (int e = tid; e < M * M; e += nthr) sS[e] = Gb[e];
              __syncthreads();
              for (int e = tid; e < M * M; e += nthr) {
                const int a = e / M, b = e - a * M;
                cf acc = czero();
                for (int c = 0; c < M; ++c) cacc_cb(acc, ld4(sS[a * M + c]), ld4(sQa[b * M + c]));
                cnorm(acc);
                sT[e] = st4(acc);
              }
              __syncthreads();
              for (int e = tid; e < M * M; e += nthr) {
                const double2 gv = to_d2(ld4(sS[e])), bv = to_d2(ld4(sQb[e]));
                acc_mu -= wk * fma(gv.x, bv.x, gv.y * bv.y);
              }
            }
            double2* out = p.gq + ((int64_t)(it.g - p.gb0) * p.n_iw + n) * p.mmax * p.mmax;
            const double cb = nbar * 2.0 / beta;
            for (int e = tid; e < M * M; e += nthr) {
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
      }
      if (p.mode & kOcc) {
        const double tr_ = block_sum_any(acc_tr, s_red);
        const double g2 = block_sum_any((double)g2h + (double)g2l, s_red);
        if (tid == 0) {
          double* o = p.occ_part + ((int64_t)kk * p.n_chunks + it.chunk) * 2;
          o[0] = tr_;
          o[1] = g2;
        }
      }
      if (p.mode & kAdj) {
        const double mb = block_sum_any(acc_mu, s_red);
        if (tid == 0) p.mubar_part[(int64_t)kk * p.n_chunks + it.chunk] = mb;
      }
      __syncthreads();
    }
  }
}

// Tile shapes: (RA, RB), the thread bound of the instantiation, and the
// largest window each serves (TR = ceil(N / RA), TC = ceil(N / RB), TR * TC <= MAXT).
struct Shape {
  int ra, rb, maxt, nmax;
};
constexpr Shape kShapes[] = {
    {1, 1, 512, 8}, {2, 2, 512, 16}, {2, 5, 512, 40}, {4, 4, 512, 64}, {3, 7, 512, 96},
};
constexpr int kNumShapes = (int)(sizeof(kShapes) / sizeof(kShapes[0]));

template <int RA, int RB, int MAXT, int MINB>
cudaError_t launch_r(const PointParams& p, int grid, int threads, size_t smem, cudaStream_t s) {
  if (threads > MAXT) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_point_df64r<RA, RB, MAXT, MINB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_point_df64r<RA, RB, MAXT, MINB><<<grid, threads, smem, s>>>(p);
  return cudaGetLastError();
}

template <int RA, int RB, int MAXT, int MINB>
int bps_r(int threads, size_t smem) {
  int nb = 0;
  cudaFuncSetAttribute(k_point_df64r<RA, RB, MAXT, MINB>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_point_df64r<RA, RB, MAXT, MINB>, threads,
                                                    smem) != cudaSuccess)
    return 0;
  return nb;
}

}  // namespace

int df64r_shape(int nbmax) {
  for (int i = 0; i < kNumShapes; ++i)
    if (nbmax <= kShapes[i].nmax) return i;
  return -1;
}

int df64r_num_shapes() { return kNumShapes; }

int df64r_tile(int shape, int which) {
  if (shape < 0 || shape >= kNumShapes) return 0;
  return which == 0 ? kShapes[shape].ra : kShapes[shape].rb;
}

bool df64r_shape_fits(int shape, int nbmax) {
  if (shape < 0 || shape >= kNumShapes) return false;
  const Shape sh = kShapes[shape];
  return ((nbmax + sh.ra - 1) / sh.ra) * ((nbmax + sh.rb - 1) / sh.rb) <= sh.maxt;
}

int df64r_threads(int shape, int nbmax) {
  const Shape sh = kShapes[shape];
  const int t = ((nbmax + sh.ra - 1) / sh.ra) * ((nbmax + sh.rb - 1) / sh.rb);
  return 32 + ((t + 31) / 32) * 32;  // owners plus the pivot warp
}

size_t point_df64r_smem(int nbmax, int mmax, int mode) {
  return make_layout_r(nbmax, mmax, mode).bytes;
}

int point_df64r_blocks_per_sm(int shape, int threads, size_t smem) {
  switch (shape) {
    case 0: return bps_r<1, 1, 512, 1>(threads, smem);
    case 1: return bps_r<2, 2, 512, 1>(threads, smem);
    case 2: return bps_r<2, 5, 512, 1>(threads, smem);
    case 3: return bps_r<4, 4, 512, 1>(threads, smem);
    case 4: return bps_r<3, 7, 512, 1>(threads, smem);
  }
  return 0;
}

cudaError_t launch_point_df64r(int shape, const PointParams& p, int grid, int threads, size_t smem,
                               cudaStream_t s) {
  switch (shape) {
    case 0: return launch_r<1, 1, 512, 1>(p, grid, threads, smem, s);
    case 1: return launch_r<2, 2, 512, 1>(p, grid, threads, smem, s);
    case 2: return launch_r<2, 5, 512, 1>(p, grid, threads, smem, s);
    case 3: return launch_r<4, 4, 512, 1>(p, grid, threads, smem, s);
    case 4: return launch_r<3, 7, 512, 1>(p, grid, threads, smem, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace gf

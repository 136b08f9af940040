// One warp, one matrix: the FP32 embedding and Gauss-Jordan inverse of the mixed path's
// warp kernels (device code only).  Used by the N(mu) kernel k_point_w32 and by the
// fused kernel k_point_f32w, whose warps invert one frequency each before the CTA runs
// the refined projections.
//
// A = (i w_n + mu) I - H_k - P_k^+ T with T = Sigma(i w_n) P_k (Eq. dmftloop1), FP32,
// the diagonal (i w_n + mu - H_ii) formed in FP64 and rounded once (warp_point_inputs).
//
// Layout: lane l holds row l (NMAX complex registers).  Windows of 33 to 40 bands add
// rows 32 to 39, each split over a group of four lanes: lane l holds columns
// 10 (l mod 4) to 10 (l mod 4) + 9 of row 32 + l / 4, so every lane updates 50 entries
// per pivot instead of the 80 of two whole rows a lane.
//
// Gauss-Jordan in exchange form with partial pivoting, every register index static
// (each step rotates the rows by one column, so the pivot column is register 0; a split
// row rotates across its four lanes with one shuffle), and lazy row scaling: the stored
// matrix is the true one with each former pivot row divided by its scale s_p.  Step j,
// pivot row p (unused, largest max(|Re|, |Im|)), u = row p as stored (its scale is still
// 1), r = 1 / u_j:
//   every other row i:  l_i = a_ij r;  a_ic -= l_i u_c (c != j);  a_ij = -l_i
//   row p:              unchanged except a_pj = 1, and its scale becomes r
// which is the sweep of the true matrix written in stored terms (a former pivot row
// updates with its stored values, because its true l and its true entries carry the
// same scale).  The pivot row reaches the warp through a shared-memory buffer, the pivot
// through a warp max-reduction; the true inverse is s_r a_rc at the end.
#pragma once

#include "gf_complex.cuh"
#include "gf_internal.cuh"

namespace gf {
namespace wgj {

using namespace cx;

__device__ __forceinline__ float2 zero2() { return make_float2(0.f, 0.f); }

// Pivot key with the row index in its low 7 bits: the largest key wins, ties go to the
// lowest row.
__device__ __forceinline__ unsigned pack_key_w(float2 v, int i) {
  return (pivot_key_s(v) & ~127u) | (unsigned)(127 - i);
}

// The warp's shared-memory region: T = Sigma P on entry (M x N, row stride N), the
// inverse B on exit (N x ld, ld = N | 1); the pivot-row buffer (NMAX entries, 16-byte
// aligned); the pivot tables p, q = p^{-1} and the row offsets p_i ld (NMAX each).
struct WarpBufs {
  float2* sX;
  float2* sBuf;
  int* sPiv;
  int* sIdx;
  int* sRow;
};

// Per-frequency inputs of one warp's matrix: Sigma(i w_n) (Sn, M x M, FP32) to sS, the
// diagonal (i w_n + mu - H_ii) formed in FP64 and rounded once to sD, and T = Sigma P
// (M x N) to sX; visible to the whole warp on return.
__device__ __forceinline__ void warp_point_inputs(const float2* __restrict__ Sn, const double2* sHii,
                                                  const float2* sP, double mu, double wn, int N, int M, int lane,
                                                  float2* sS, float2* sD, float2* sX) {
  for (int e = lane; e < M * M; e += 32) sS[e] = Sn[e];
  for (int x = lane; x < N; x += 32)
    sD[x] = make_float2(__double2float_rn(mu - sHii[x].x), __double2float_rn(wn - sHii[x].y));
  __syncwarp();
  for (int e = lane; e < M * N; e += 32) {
    const int a = e / N, j = e - a * N;
    float2 acc = zero2();
    for (int b = 0; b < M; ++b) fmac(acc, sS[a * M + b], sP[b * N + j]);
    sX[e] = acc;
  }
  __syncwarp();
}

// Embedding, elimination and the inverse in shared memory, for N <= NMAX (SPLIT: NMAX =
// 40 and rows 32 to 39 split).  On exit X[i][c] = sX[sRow[i] + sIdx[c]], visible to the
// whole warp.  Hk: H_k in FP32 (N x N); sD: the diagonal; sP: P_k in FP32 (M x N).
template <int NMAX, bool SPLIT>
__device__ __forceinline__ void warp_invert(const float2* __restrict__ Hk, const float2* sD, const float2* sP,
                                            const WarpBufs& b, int N, int M, int lane, int* status) {
  static_assert(!SPLIT || NMAX == 40, "split rows: windows of 33 to 40 bands");
  constexpr int SEG = NMAX / 4;  // columns of a split row on one lane
  const int ld = N | 1;
  // split row of this lane: row 32 + lane / 4, columns c1 .. c1 + SEG - 1 (register order)
  const int g = lane & 3, r1 = 32 + (lane >> 2), c1 = SEG * g;
  const int lead = lane & ~3, nxt = lead | ((lane + 1) & 3);
  float2* sX = b.sX;
  float2* sBuf = b.sBuf;
  // A = diag - H - P^+ T: row lane, and the split row's segment
  float2 a[NMAX];
  float2 a1[SPLIT ? SEG : 1];
#pragma unroll
  for (int c = 0; c < NMAX; ++c) {
    float2 v = zero2();
    if (lane < N && c < N) {
      const float2 h = Hk[lane * N + c];
      v = (lane == c) ? sD[lane] : make_float2(-h.x, -h.y);
    }
    a[c] = v;
  }
  if (lane < N) {
    for (int x = 0; x < M; ++x) {
      const float2 pv = sP[x * N + lane];
      const float2 mp = make_float2(-pv.x, pv.y);  // -conj(P[x][lane])
#pragma unroll
      for (int c = 0; c < NMAX; ++c)
        if (c < N) fmac(a[c], mp, sX[x * N + c]);
    }
  }
  if constexpr (SPLIT) {
#pragma unroll
    for (int y = 0; y < SEG; ++y) {
      const int c = c1 + y;
      float2 v = zero2();
      if (r1 < N && c < N) {
        const float2 h = Hk[r1 * N + c];
        v = (r1 == c) ? sD[r1] : make_float2(-h.x, -h.y);
      }
      a1[y] = v;
    }
    if (r1 < N) {
      for (int x = 0; x < M; ++x) {
        const float2 pv = sP[x * N + r1];
        const float2 mp = make_float2(-pv.x, pv.y);
#pragma unroll
        for (int y = 0; y < SEG; ++y)
          if (c1 + y < N) fmac(a1[y], mp, sX[x * N + c1 + y]);
      }
    }
  }
  // Gauss-Jordan, lazy row scales.  Each step rotates every row left by one column, so
  // the pivot column is always register 0 and the loop body stays small; after step j
  // the original column c sits at register (c - j - 1) mod NMAX.
  bool used = false, used1 = false;
  float2 sc = make_float2(1.f, 0.f), sc1 = make_float2(1.f, 0.f);
#pragma unroll 1
  for (int j = 0; j < N; ++j) {
    unsigned key = (lane < N && !used) ? pack_key_w(a[0], lane) : 0u;
    // a split row's pivot-column entry sits on the first lane of its group
    if constexpr (SPLIT)
      if (g == 0 && r1 < N && !used1) key = max(key, pack_key_w(a1[0], r1));
    const unsigned best = __reduce_max_sync(0xffffffffu, key);
    if (lane == 0 && ((best >> 7) == 0u || (best & ~127u) >= 0x7f800000u)) atomicOr(status, kFlagSingular);
    const int prow = min(127 - (int)(best & 127u), N - 1);
    if (lane == prow)
#pragma unroll
      for (int c = 0; c < NMAX; ++c) sBuf[c] = a[c];
    if constexpr (SPLIT)
      if (r1 == prow)
#pragma unroll
        for (int y = 0; y < SEG; ++y) sBuf[c1 + y] = a1[y];
    __syncwarp();
    const float2 r = frcp(sBuf[0]);
    const bool isp = (lane == prow);
    const float2 lq = isp ? zero2() : fmul(a[0], r);
#pragma unroll
    for (int c = 1; c < NMAX; ++c) {
      const float2 uc = sBuf[c];
      fsub_prod(a[c], lq, uc);
    }
    {
      const float2 col = isp ? make_float2(1.f, 0.f) : make_float2(-lq.x, -lq.y);
#pragma unroll
      for (int c = 0; c + 1 < NMAX; ++c) a[c] = a[c + 1];
      a[NMAX - 1] = col;
      if (isp) {
        used = true;
        sc = r;
      }
    }
    if constexpr (SPLIT) {
      // the split row: l from its first lane; every entry updated (the pivot column's
      // is replaced below), then the row rotates left across the group
      const float2 h1 = make_float2(__shfl_sync(0xffffffffu, a1[0].x, lead),
                                    __shfl_sync(0xffffffffu, a1[0].y, lead));
      const bool isp1 = (r1 == prow);
      const float2 lq1 = isp1 ? zero2() : fmul(h1, r);
#pragma unroll
      for (int y = 0; y < SEG; ++y) fsub_prod(a1[y], lq1, sBuf[c1 + y]);
      if (g == 0) a1[0] = isp1 ? make_float2(1.f, 0.f) : make_float2(-lq1.x, -lq1.y);
      const float2 t = make_float2(__shfl_sync(0xffffffffu, a1[0].x, nxt),
                                   __shfl_sync(0xffffffffu, a1[0].y, nxt));
#pragma unroll
      for (int y = 0; y + 1 < SEG; ++y) a1[y] = a1[y + 1];
      a1[SEG - 1] = t;
      if (isp1) {
        used1 = true;
        sc1 = r;
      }
    }
    if (lane == 0) b.sPiv[j] = prow;
    __syncwarp();  // the buffer is rewritten by the next pivot
  }
  // the inverse (true values s_r a_rc): X[i][c] = B[p_i][q_c]; register x holds the
  // original column (x + N) mod NMAX
  if (lane < N)
#pragma unroll
    for (int x = 0; x < NMAX; ++x) {
      int c = x + N;
      if (c >= NMAX) c -= NMAX;
      if (c < N) sX[lane * ld + c] = fmul(sc, a[x]);
    }
  if constexpr (SPLIT)
    if (r1 < N)
#pragma unroll
      for (int y = 0; y < SEG; ++y) {
        int c = c1 + y + N;
        if (c >= NMAX) c -= NMAX;
        if (c < N) sX[r1 * ld + c] = fmul(sc1, a1[y]);
      }
  __syncwarp();
  for (int j = lane; j < N; j += 32) b.sIdx[b.sPiv[j]] = j;
  __syncwarp();
  for (int x = lane; x < N; x += 32) b.sRow[x] = b.sPiv[x] * ld;
  __syncwarp();
}

}  // namespace wgj
}  // namespace gf
